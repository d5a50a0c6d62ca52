"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws the inputs.  The paper evaluates
FlexProofs on uniformly random vectors of N = 2^16 .. 2^24 field elements (Sec. 5.2); the
generators below reproduce that shape.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) -- state advances by 0x9e3779b97f4a7c15 and each output is the
MurmurHash3 variant-13 finaliser of the state.  Output k of the stream seeded with s is
therefore mix(s + (k + 1) * gamma) mod 2^64, which is what the vectorised form computes.

An Fr value is drawn from four consecutive outputs (little-endian 64-bit limbs, the top limb
masked to 63 bits) and rejected while >= r, so the accepted values are uniform in [0, r).
"""
from __future__ import annotations

import math
import numpy as np

# BLS12-381 scalar field modulus r, as four little-endian 64-bit limbs.
R_LIMBS = (0xFFFFFFFF00000001, 0x53BDA402FFFE5BFE, 0x3339D80809A1D805, 0x73EDA753299D7D48)
R_INT = sum(v << (64 * i) for i, v in enumerate(R_LIMBS))

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream seeded with `seed`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & (2**64 - 1)) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _below_r(c: np.ndarray) -> np.ndarray:
    lt = np.zeros(len(c), dtype=bool)
    eq = np.ones(len(c), dtype=bool)
    for limb in (3, 2, 1, 0):
        rl = np.uint64(R_LIMBS[limb])
        lt |= eq & (c[:, limb] < rl)
        eq &= c[:, limb] == rl
    return lt


def fr_uniform(seed: int, n: int) -> np.ndarray:
    """n uniform Fr elements, shape (n, 4) uint64, little-endian canonical limbs."""
    out = np.empty((0, 4), dtype=np.uint64)
    cand0 = 0
    while len(out) < n:
        need = n - len(out)
        ncand = int(need * 1.12) + 64
        raw = splitmix64(seed, 4 * cand0, 4 * ncand).reshape(ncand, 4).copy()
        raw[:, 3] &= np.uint64(0x7FFFFFFFFFFFFFFF)
        keep = raw[_below_r(raw)]
        out = np.concatenate([out, keep[:need]])
        cand0 += ncand
    return np.ascontiguousarray(out)


def u32_embedded(seed: int, n: int) -> np.ndarray:
    """n uniform 32-bit integers embedded in Fr (value distribution (b) of the N=2^16 workload)."""
    out = np.zeros((n, 4), dtype=np.uint64)
    out[:, 0] = splitmix64(seed, 0, n) & np.uint64(0xFFFFFFFF)
    return out


def vector(seed: int, log_n: int, dist: str = "uniform") -> np.ndarray:
    n = 1 << log_n
    if dist == "uniform":
        return fr_uniform(seed, n)
    if dist == "u32":
        return u32_embedded(seed, n)
    raise ValueError(dist)


def to_ints(m: np.ndarray) -> list[int]:
    m = np.asarray(m, dtype=np.uint64)
    return [int(a) | (int(b) << 64) | (int(c) << 128) | (int(d) << 192) for a, b, c, d in m]


def nearest_pow2(x: int) -> int:
    """Nearest power of two by linear distance (ties would round down; none occur for k in 8..18)."""
    lo = 1 << (x.bit_length() - 1)
    hi = lo << 1
    return lo if x - lo <= hi - x else hi


def batched_jobs(seed: int, njobs: int = 64, kmin: int = 8, kmax: int = 18):
    """The 64-job batched workload: k uniform in [kmin, kmax] by seed, N = 2^k,
    b = min(R, nearest power of two to k^2), job j's vector drawn from seed + 1 + j."""
    ks = splitmix64(seed, 0, njobs) % np.uint64(kmax - kmin + 1) + np.uint64(kmin)
    jobs = []
    for j, k in enumerate(ks.tolist()):
        R = 1 << (k // 2)
        jobs.append({"log_n": int(k), "b": min(R, nearest_pow2(k * k)), "seed": seed + 1 + j})
    return jobs


def poisson_trace(seed: int, nreq: int = 2000, rate: float = 200.0, kmin: int = 10, kmax: int = 20,
                  bs=(1, 16, 256)):
    """The served workload: exponential inter-arrivals with the given mean rate, k uniform in
    [kmin, kmax], b uniform in `bs` clamped to R."""
    u = splitmix64(seed, 0, 3 * nreq).reshape(nreq, 3)
    t = 0.0
    reqs = []
    for i in range(nreq):
        u0 = (int(u[i, 0]) >> 11) * (1.0 / (1 << 53))
        t += -math.log1p(-u0) / rate
        k = kmin + int(u[i, 1] % np.uint64(kmax - kmin + 1))
        b = bs[int(u[i, 2] % np.uint64(len(bs)))]
        R = 1 << (k // 2)
        reqs.append({"t": t, "log_n": k, "b": min(b, R), "seed": seed + 1 + i})
    return reqs
