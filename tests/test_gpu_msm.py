"""GPU parity of the batched Pippenger G1 MSM (fp_msm_g1) through the C ABI.

Exact arithmetic, zero tolerance.  Small cases compare against the oracle's naive per-term
double-and-add MSM; large cases against the closed form: with bases P_i = s_i g1,
sum_i k_i P_i = (sum_i k_i s_i mod r) g1, which pins the MSM without running one on the CPU.
Edge cases: zero scalars, repeated scalars and bases (bucket doublings), P and -P in one bucket
(cancellation to the identity), identity bases, scalars >= r and up to 2^256 - 1, n = 0, every
window size, several batches over shared bases and over consecutive slices of the bases.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402

R = I.R_INT
P_FQ = O.const_p()


def limbs(vals):
    """Python ints < 2^256 -> n x 4 little-endian uint64."""
    out = np.zeros((len(vals), 4), np.uint64)
    for i, v in enumerate(vals):
        for w in range(4):
            out[i, w] = (v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF
    return out


@functools.lru_cache(maxsize=None)
def base_scalars(seed, n):
    return I.to_ints(I.fr_uniform(seed, n))


@functools.lru_cache(maxsize=None)
def oracle_points(seed, n):
    g = O.g1_gen()
    return tuple(O.g1_mul(g, s) for s in base_scalars(seed, n))


def closed_form(s, k):
    return O.g1_mul(O.g1_gen(), sum(a * b for a, b in zip(s, k)) % R)


def closed_form_np(s_np, k_np):
    """closed_form for n x 4 little-endian uint64 arrays, read element by element from the bytes."""
    ms, mk = memoryview(s_np.tobytes()), memoryview(k_np.tobytes())
    fb = int.from_bytes
    dot = sum(fb(ms[o:o + 32], "little") * fb(mk[o:o + 32], "little") for o in range(0, len(ms), 32))
    return O.g1_mul(O.g1_gen(), dot % R)


def neg_point(p: bytes) -> bytes:
    if p == bytes(96):
        return p
    y = int.from_bytes(p[48:], "big")
    return p[:48] + ((P_FQ - y) % P_FQ).to_bytes(48, "big")


@pytest.mark.parametrize("window", [0, 4, 5, 7, 9, 11, 13, 16])
def test_msm_vs_oracle_naive(window):
    n = 203                                            # ragged: not a multiple of any tile
    pts = oracle_points(11, n)
    k = base_scalars(12, n)
    bases = F.G1Bases(scalars=limbs(base_scalars(11, n)))
    got = F.msm_g1(bases, limbs(k), 1, window)
    assert got == O.g1_msm(b"".join(pts), list(k))


def test_msm_edge_scalars_and_bases():
    n = 64
    pts = list(oracle_points(21, n))
    pts[5] = bytes(96)                                 # identity base
    pts[7] = neg_point(pts[6])                         # P and -P
    pts[9] = pts[8]                                    # repeated base
    k = list(base_scalars(22, n))
    k[0] = 0
    k[1] = 1
    k[2] = R - 1
    k[3] = R                                           # >= r: integer combination
    k[4] = (1 << 256) - 1
    k[6] = k[7] = 123456789                            # P and -P with equal scalars cancel
    k[8] = k[9] = 987654321                            # same bucket twice: doubling inside a bucket
    for i in range(40, 50):
        k[i] = 5                                       # many entries in one bucket
    bases = F.G1Bases(points=b"".join(pts))
    for window in (4, 8, 16):
        assert F.msm_g1(bases, limbs(k), 1, window) == O.g1_msm(b"".join(pts), k)


def test_msm_all_zero_and_empty():
    bases = F.G1Bases(scalars=limbs(base_scalars(31, 16)))
    assert F.msm_g1(bases, limbs([0] * 16), 1, 0) == bytes(96)
    assert F.msm_g1(bases, np.zeros((0, 4), np.uint64), 3, 0) == bytes(3 * 96)


def test_msm_bad_points_rejected():
    p = bytearray(oracle_points(41, 2)[0])
    p[95] ^= 1                                         # off the curve
    with pytest.raises(F.FlexProofsError) as e:
        F.G1Bases(points=bytes(p))
    assert e.value.status == 1
    big = P_FQ.to_bytes(48, "big") + bytes(48)         # x = p is not canonical
    with pytest.raises(F.FlexProofsError):
        F.G1Bases(points=big)
    with pytest.raises(F.FlexProofsError):            # on the curve, outside the order-r subgroup
        F.G1Bases(points=off_subgroup_point())


def off_subgroup_point() -> bytes:
    """The first (x, y) on y^2 = x^3 + 4 with x = 1, 2, ...: the cofactor h1 ~ 2^126 leaves it
    outside G1 (checked here by [r] P != 0 with the oracle)."""
    for x in range(1, 100):
        rhs = (x ** 3 + 4) % P_FQ
        y = pow(rhs, (P_FQ + 1) // 4, P_FQ)                # p = 3 mod 4
        if y * y % P_FQ == rhs:
            pt = x.to_bytes(48, "big") + y.to_bytes(48, "big")
            assert O.g1_valid(pt) and O.g1_mul(pt, R) != bytes(96)
            return pt
    raise AssertionError("no point found")


@pytest.mark.parametrize("window", [0, 6, 12])
def test_msm_batches_shared_and_sliced(window):
    n, nb = 50, 3
    s = base_scalars(51, n * nb)
    k = base_scalars(52, n * nb)
    shared = F.G1Bases(scalars=limbs(s[:n]))
    got = F.msm_g1(shared, limbs(k), nb, window)
    for j in range(nb):
        assert got[96 * j: 96 * (j + 1)] == closed_form(s[:n], k[j * n:(j + 1) * n])
    sliced = F.G1Bases(scalars=limbs(s))
    got = F.msm_g1(sliced, limbs(k), nb, window)
    for j in range(nb):
        assert got[96 * j: 96 * (j + 1)] == closed_form(s[j * n:(j + 1) * n], k[j * n:(j + 1) * n])


def test_msm_device_path_matches_host():
    n, nb = 1000, 2
    s = base_scalars(61, n)
    k = limbs(base_scalars(62, n * nb))
    bases = F.G1Bases(scalars=torch.from_numpy(limbs(s).view(np.int64)).cuda())
    kd = torch.from_numpy(k.view(np.int64)).cuda()
    out = torch.zeros(96 * nb, dtype=torch.uint8, device="cuda")
    F.msm_g1(bases, kd, nb, 0, torch.cuda.current_stream(), out)
    torch.cuda.synchronize()
    assert bytes(out.cpu().numpy()) == F.msm_g1(bases, k, nb, 0)


def test_msm_naive_n4096():
    """2^12 terms (the smallest size of the MSM sweep, autotuned window) against the oracle's naive
    per-term double-and-add MSM."""
    n = 1 << 12
    pts = oracle_points(13, n)
    k = base_scalars(14, n)
    bases = F.G1Bases(scalars=limbs(base_scalars(13, n)))
    assert F.msm_g1(bases, limbs(k), 1, 0) == O.g1_msm(b"".join(pts), list(k))


@pytest.mark.parametrize("log_n", [12, 16, 20, 24])
def test_msm_closed_form_large(log_n):
    """Sizes of the MSM sweep (2^24: its largest); the autotuner's choice is exercised at 2^16."""
    n = 1 << log_n
    s_np = I.fr_uniform(70 + log_n, n)
    k_np = I.fr_uniform(80 + log_n, n)
    bases = F.G1Bases(scalars=torch.from_numpy(s_np.view(np.int64)).cuda())
    kd = torch.from_numpy(k_np.view(np.int64)).cuda()
    if log_n == 16:
        c, ms = F.msm_autotune(bases, kd, 1)
        assert 4 <= c <= 16 and ms > 0 and F.msm_window(n, 1) == c
    out = torch.zeros(96, dtype=torch.uint8, device="cuda")
    F.msm_g1(bases, kd, 1, 0, None, out)
    torch.cuda.synchronize()
    assert bytes(out.cpu().numpy()) == closed_form_np(s_np, k_np)
