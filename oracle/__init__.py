"""FlexProofs CPU oracle (ctypes binding) -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of the FlexProofs ProveAll path (arXiv 2601.03031, Sec. 2-4 and
Appendix C) written in C (``oracle/*.c``).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with the CUDA path.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  - Fq/Fr/Fq2/Fq12 arithmetic, constants: pinned (Python integers, derivation from x).
  - SHA-256: pinned (hashlib).  HFr, SplitMix64: pinned (Python re-derivation from their
    published definitions; the tag/concatenation layout itself is a reading, see below).
  - G1/G2 group law and scalar multiplication: pinned (brute force, group order, closed forms).
  - Pairing: pinned by bilinearity, non-degeneracy, order r and an independent
    from-the-definition Miller function in pure Python.
  - PST / FC / VC: pinned by trapdoor closed forms, the FC round invariant, brute-force
    ProveOne, every proof verifying, tamper rejection and the paper's proof-size formula.
  - Absolute bytes of Fiat-Shamir and Merkle outputs (r_a, x_j, z, every digest, r_j, every
    proof byte): pinned by an independent pure-Python re-derivation from hashlib, HFr and the
    known discrete logarithms (tests/test_oracle_transcript.py), which also checks that changing
    any one encoding reading is detected.  The readings themselves are choices where the paper
    leaves the random oracles and the Merkle instantiation open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["fields.c", "curves.c", "hash.c", "vc.c", "api.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable C11, no intrinsics)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(p) for p in srcs + [hdr])
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + srcs)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_u8p = ctypes.c_char_p
            vp = ctypes.c_void_p
            L.or_setup.restype = vp
            L.or_setup.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
            L.or_setup_split.restype = vp
            L.or_setup_split.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
            L.or_segment_proof_len.restype = ctypes.c_size_t
            L.or_segment_proof_len.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
            L.or_verify_segment.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp, ctypes.c_size_t]
            L.or_eval_proof_len.restype = ctypes.c_size_t
            L.or_eval_proof_len.argtypes = [vp]
            L.or_eval_prove.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_eval_verify.argtypes = [vp, vp, vp, vp, ctypes.c_size_t]
            L.or_pp_free.argtypes = [vp]
            L.or_pp_bytes.restype = ctypes.c_size_t
            L.or_pp_bytes.argtypes = [vp, vp]
            L.or_pp_info.argtypes = [vp, vp]
            L.or_pp_trapdoor.argtypes = [vp, vp]
            L.or_commit.argtypes = [vp, vp, vp, vp]
            L.or_bopen_len.restype = ctypes.c_size_t
            L.or_bopen_len.argtypes = [vp]
            L.or_bopen.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_int]
            L.or_prover_new.restype = vp
            L.or_prover_new.argtypes = [vp, vp, vp, vp, ctypes.c_uint32]
            L.or_prover_free.argtypes = [vp]
            L.or_prover_block.argtypes = [vp, ctypes.c_uint32]
            L.or_prover_block_bytes.restype = vp
            L.or_prover_block_bytes.argtypes = [vp, ctypes.c_uint32]
            L.or_prover_step2.argtypes = [vp]
            L.or_proof_len.restype = ctypes.c_size_t
            L.or_proof_len.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
            L.or_prover_proof.argtypes = [vp, ctypes.c_uint64, vp, ctypes.c_size_t, vp]
            L.or_prover_step2_parts.argtypes = [vp, vp, vp, vp, vp]
            L.or_prover_state.restype = ctypes.c_size_t
            L.or_prover_state.argtypes = [vp, vp]
            L.or_prove_one.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_uint64, vp, ctypes.c_size_t, vp]
            L.or_verify.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint64, vp, vp, ctypes.c_size_t, ctypes.c_int]
            L.or_const.argtypes = [ctypes.c_int, vp]
            L.or_fq_op.argtypes = [ctypes.c_int, vp, vp, vp]
            L.or_fr_op.argtypes = [ctypes.c_int, vp, vp, vp]
            L.or_fq2_mul.argtypes = [vp, vp, vp]
            L.or_fr_wide.argtypes = [vp, ctypes.c_int, vp]
            L.or_fq12_mul.argtypes = [vp, vp, vp]
            L.or_fq12_pow.argtypes = [vp, vp, ctypes.c_int, vp]
            L.or_fq12_conj.argtypes = [vp, vp]
            for n in ("or_g1_gen", "or_g2_gen"):
                getattr(L, n).argtypes = [vp]
            for n in ("or_g1_mul", "or_g1_add", "or_g2_mul", "or_g2_add", "or_pairing", "or_miller"):
                getattr(L, n).argtypes = [vp, vp, vp]
            L.or_g1_dbl.argtypes = [vp, vp]
            L.or_final_exp.argtypes = [vp, vp]
            L.or_g1_valid.argtypes = [vp]
            L.or_g2_valid.argtypes = [vp]
            L.or_g1_msm.argtypes = [vp, vp, ctypes.c_uint32, vp]
            L.or_sha256.argtypes = [vp, ctypes.c_size_t, vp]
            L.or_hfr.argtypes = [c_u8p, vp, ctypes.c_size_t, vp]
            L.or_splitmix_fr.argtypes = [ctypes.c_uint64, ctypes.c_uint32, vp]
            L.or_ops_reset.argtypes = []
            L.or_ops_reset.restype = None
            L.or_ops_get.argtypes = [vp]
            L.or_ops_get.restype = None
            rc = L.or_status()
            if rc != 0:
                raise RuntimeError(f"oracle constant derivation failed: {rc}")
            _lib = L
    return _lib


def _buf(n: int):
    return ctypes.create_string_buffer(n)


def _call(fn, *args):
    rc = fn(*args)
    if rc != 0:
        raise ValueError(f"{fn.__name__} failed ({rc})")


# --------------------------------------------------------------------------- constants
def const_p() -> int:
    b = _buf(48); lib().or_const(0, b); return int.from_bytes(b.raw, "big")


def const_r() -> int:
    b = _buf(32); lib().or_const(1, b); return int.from_bytes(b.raw, "big")


def const_final_exp() -> int:
    b = _buf(4 * 160); n = lib().or_const(2, b)
    return int.from_bytes(b.raw[: 4 * n], "little")


# --------------------------------------------------------------------------- operation counts
def ops_reset() -> None:
    """Zero the counters of Miller loops, final exponentiations and G1 / G2 scalar multiplications."""
    lib().or_ops_reset()


def ops() -> dict:
    """Operations since the last ops_reset() (all threads)."""
    a = (ctypes.c_uint64 * 4)()
    lib().or_ops_get(a)
    return {"miller": a[0], "final_exp": a[1], "g1_mul": a[2], "g2_mul": a[3]}


# --------------------------------------------------------------------------- fields
def fq_op(op: str, a: int, b: int = 0) -> int:
    o = _buf(48)
    _call(lib().or_fq_op, {"add": 0, "sub": 1, "mul": 2, "inv": 3}[op], a.to_bytes(48, "big"), b.to_bytes(48, "big"), o)
    return int.from_bytes(o.raw, "big")


def fr_op(op: str, a: int, b: int = 0) -> int:
    o = _buf(32)
    _call(lib().or_fr_op, {"add": 0, "sub": 1, "mul": 2, "inv": 3}[op], a.to_bytes(32, "big"), b.to_bytes(32, "big"), o)
    return int.from_bytes(o.raw, "big")


def fq2_mul(a, b):
    o = _buf(96)
    _call(lib().or_fq2_mul, a[0].to_bytes(48, "big") + a[1].to_bytes(48, "big"),
          b[0].to_bytes(48, "big") + b[1].to_bytes(48, "big"), o)
    return int.from_bytes(o.raw[:48], "big"), int.from_bytes(o.raw[48:], "big")


def fr_from_wide(data: bytes) -> int:
    o = _buf(32); lib().or_fr_wide(data, len(data), o); return int.from_bytes(o.raw, "big")


def fq12_mul(a: bytes, b: bytes) -> bytes:
    o = _buf(576); _call(lib().or_fq12_mul, a, b, o); return o.raw


def fq12_pow(a: bytes, e: int) -> bytes:
    nw = max(1, (e.bit_length() + 31) // 32)
    ew = e.to_bytes(4 * nw, "little")
    o = _buf(576); _call(lib().or_fq12_pow, a, ew, nw, o); return o.raw


def fq12_conj(a: bytes) -> bytes:
    o = _buf(576); _call(lib().or_fq12_conj, a, o); return o.raw


# --------------------------------------------------------------------------- groups
def g1_gen() -> bytes:
    o = _buf(96); _call(lib().or_g1_gen, o); return o.raw


def g2_gen() -> bytes:
    o = _buf(192); _call(lib().or_g2_gen, o); return o.raw


def g1_mul(p: bytes, k: int) -> bytes:
    o = _buf(96); _call(lib().or_g1_mul, p, k.to_bytes(32, "big"), o); return o.raw


def g1_add(p: bytes, q: bytes) -> bytes:
    o = _buf(96); _call(lib().or_g1_add, p, q, o); return o.raw


def g1_dbl(p: bytes) -> bytes:
    o = _buf(96); _call(lib().or_g1_dbl, p, o); return o.raw


def g2_mul(p: bytes, k: int) -> bytes:
    o = _buf(192); _call(lib().or_g2_mul, p, k.to_bytes(32, "big"), o); return o.raw


def g2_add(p: bytes, q: bytes) -> bytes:
    o = _buf(192); _call(lib().or_g2_add, p, q, o); return o.raw


def g1_valid(p: bytes) -> bool:
    return bool(lib().or_g1_valid(p))


def g2_valid(p: bytes) -> bool:
    return bool(lib().or_g2_valid(p))


def g1_msm(points: bytes, scalars: list[int]) -> bytes:
    ks = b"".join(k.to_bytes(32, "big") for k in scalars)
    o = _buf(96); _call(lib().or_g1_msm, points, ks, len(scalars), o); return o.raw


def pairing(p: bytes, q: bytes) -> bytes:
    o = _buf(576); _call(lib().or_pairing, p, q, o); return o.raw


def miller(p: bytes, q: bytes) -> bytes:
    o = _buf(576); _call(lib().or_miller, p, q, o); return o.raw


def final_exp(f: bytes) -> bytes:
    o = _buf(576); _call(lib().or_final_exp, f, o); return o.raw


# --------------------------------------------------------------------------- hashing
def sha256(msg: bytes) -> bytes:
    o = _buf(32); lib().or_sha256(msg, len(msg), o); return o.raw


def hfr(tag: str, data: bytes) -> int:
    o = _buf(32); _call(lib().or_hfr, tag.encode(), data, len(data), o); return int.from_bytes(o.raw, "big")


def splitmix_fr(seed: int, n: int) -> list[int]:
    arr = (ctypes.c_uint64 * (4 * n))()
    _call(lib().or_splitmix_fr, seed, n, arr)
    return [arr[4 * i] | (arr[4 * i + 1] << 64) | (arr[4 * i + 2] << 128) | (arr[4 * i + 3] << 192) for i in range(n)]


# --------------------------------------------------------------------------- protocol
class PP:
    """VC.Setup output (Eq. vcpp) held by the oracle.  log_r (default floor(log_n / 2)) sets the
    number of segments R = 2^log_r, each of M = N / R elements (OpenAll for sub-arrays, Sec. 4.4)."""

    def __init__(self, log_n: int, seed: int, log_r: int | None = None):
        if log_r is None:
            self.h = lib().or_setup(log_n, seed)
        else:
            self.h = lib().or_setup_split(log_r, log_n - log_r, seed)
        if not self.h:
            raise ValueError("or_setup failed")
        info = (ctypes.c_uint32 * 4)()
        lib().or_pp_info(self.h, info)
        self.log_n, self.R, self.M, self.log_c = info[0], info[1], info[2], info[3]
        self.log_r = self.log_n - self.log_c
        self.N = self.R * self.M

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.or_pp_free(h)
            self.h = None

    def to_bytes(self) -> bytes:
        n = lib().or_pp_bytes(self.h, None)
        o = _buf(n); lib().or_pp_bytes(self.h, o); return o.raw

    def trapdoor(self):
        o = _buf(32 * (self.log_c + 1)); lib().or_pp_trapdoor(self.h, o)
        vals = [int.from_bytes(o.raw[32 * i: 32 * i + 32], "big") for i in range(self.log_c + 1)]
        return vals[0], vals[1:]

    def bopen_len(self) -> int:
        return lib().or_bopen_len(self.h)

    def proof_len(self, b: int, k: int) -> int:
        return lib().or_proof_len(self.h, b, k)

    def segment_proof_len(self, b: int, k: int) -> int:
        return lib().or_segment_proof_len(self.h, b, k)


def commit(pp: PP, m_limbs: bytes):
    """m_limbs: N x 4 little-endian u64 canonical Fr.  Returns (C: 576 B, rows: R*96 B)."""
    C = _buf(576); rows = _buf(96 * pp.R)
    _call(lib().or_commit, pp.h, m_limbs, C, rows)
    return C.raw, rows.raw


def bopen(pp: PP, C: bytes, rows: bytes, b: int, k: int, check_invariant: bool = False):
    o = _buf(pp.bopen_len())
    rc = lib().or_bopen(pp.h, C, rows, b, k, o, int(check_invariant))
    if rc < 0:
        raise ValueError(f"or_bopen failed ({rc})")
    return o.raw, rc == 0


class Prover:
    """OpenAll state of the oracle: Step 1 per block (threadable) and Step 2."""

    def __init__(self, pp: PP, m_limbs: bytes, C: bytes, rows: bytes, b: int):
        self.pp = pp
        self.b = b
        self.K = (pp.R + b - 1) // b
        self._keep = (m_limbs, C, rows)
        self.h = lib().or_prover_new(pp.h, m_limbs, C, rows, b)
        if not self.h:
            raise ValueError("or_prover_new failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.or_prover_free(h)
            self.h = None

    def block(self, k: int) -> None:
        _call(lib().or_prover_block, self.h, k)

    def blocks(self, ks=None, threads: int | None = None) -> None:
        ks = list(range(self.K)) if ks is None else list(ks)
        threads = threads or os.cpu_count() or 1
        if threads <= 1 or len(ks) <= 1:
            for k in ks:
                self.block(k)
            return
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(self.block, ks))

    def block_bytes(self, k: int) -> bytes:
        p = lib().or_prover_block_bytes(self.h, k)
        return ctypes.string_at(p, self.pp.bopen_len())

    def step2(self) -> None:
        _call(lib().or_prover_step2, self.h)

    def step2_parts(self):
        root = _buf(32); rj = _buf(32 * self.pp.R); gs = _buf(32 * self.pp.M); ds = _buf(96)
        lib().or_prover_step2_parts(self.h, root, rj, gs, ds)
        return root.raw, rj.raw, gs.raw, ds.raw

    def state(self) -> bytes:
        """All shared proof state (block records, Merkle trees, r_j, D_w, g_w, PST quotients) in the
        layout of the GPU library's state export; blocks not run are zeros."""
        n = lib().or_prover_state(self.h, None)
        o = _buf(n)
        if lib().or_prover_state(self.h, o) != n:
            raise ValueError("or_prover_state: Step 2 has not run")
        return o.raw

    def proof(self, i: int) -> bytes:
        k = (i // self.pp.M) // self.b
        n = self.pp.proof_len(self.b, k)
        o = _buf(n); ln = ctypes.c_size_t(0)
        _call(lib().or_prover_proof, self.h, i, o, n, ctypes.byref(ln))
        return o.raw[: ln.value]


def prove_one(pp: PP, m_limbs: bytes, C: bytes, rows: bytes, b: int, i: int) -> bytes:
    k = (i // pp.M) // b
    n = pp.proof_len(b, k)
    o = _buf(n); ln = ctypes.c_size_t(0)
    _call(lib().or_prove_one, pp.h, m_limbs, C, rows, b, i, o, n, ctypes.byref(ln))
    return o.raw[: ln.value]


def verify(pp: PP, C: bytes, b: int, i: int, m_i: int, proof: bytes, memo: bool = True) -> bool:
    """VC.Verify.  With memo=True identical FC.BVerify / PST.Verify sub-checks (same block, same
    column, byte-identical inputs) are answered from a cache keyed by a hash of those inputs."""
    return bool(lib().or_verify(pp.h, C, b, i, m_i.to_bytes(32, "big"), proof, len(proof), int(memo)))


def segment_proof(pp: PP, rows: bytes, prover: "Prover", j: int) -> bytes:
    """OpenAll for sub-arrays (Sec. 4.4): the proof of segment j is its block's row commitments and
    pi_{C_k} from Step 1 (prover.blocks() must have run for block k = j // b)."""
    b = prover.b
    k = j // b
    lo, hi = k * b, min((k + 1) * b, pp.R)
    return rows[96 * lo: 96 * hi] + prover.block_bytes(k)


def verify_segment(pp: PP, C: bytes, b: int, j: int, m_j_limbs: bytes, proof: bytes) -> bool:
    """Verifier V_j of OpenAll for sub-arrays: C_j recomputed from m_j (M x 4 little-endian u64)
    must be the block's entry j, and FC.BVerify of the block must accept."""
    return bool(lib().or_verify_segment(pp.h, C, b, j, m_j_limbs, proof, len(proof)))


def _point_bytes(pp: PP, r) -> bytes:
    assert len(r) == pp.log_n
    return b"".join(int(v).to_bytes(32, "big") for v in r)


def eval_prove(pp: PP, m_limbs: bytes, C: bytes, rows: bytes, r) -> bytes:
    """Evaluation proof of the committed vector's multilinear extension at r = (r_0 .. r_{log N - 1})
    (Sec. 4.4): y || C_F || pi_FC || pi_PST."""
    o = _buf(lib().or_eval_proof_len(pp.h))
    _call(lib().or_eval_prove, pp.h, m_limbs, C, rows, _point_bytes(pp, r), o)
    return o.raw


def eval_verify(pp: PP, C: bytes, r, proof: bytes) -> bool:
    return bool(lib().or_eval_verify(pp.h, C, _point_bytes(pp, r), proof, len(proof)))


def verify_many(pp: PP, C: bytes, b: int, items, threads: int | None = None) -> list[bool]:
    """Verify (i, m_i, proof) triples on host threads (ctypes releases the GIL)."""
    items = list(items)
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda t: verify(pp, C, b, t[0], t[1], t[2]), items))
