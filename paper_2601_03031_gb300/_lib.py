"""Thin ctypes binding of libflexproofs.so (include/flexproofs.h).  Argument marshalling only:
every step of Setup, Commit and OpenAll runs in the library's CUDA kernels.  If the library is
missing or no CUDA device is usable, calls raise -- there is no fallback path."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflexproofs.so")

FP_STATUS = {0: "FP_OK", 1: "FP_EINVAL", 2: "FP_ENOMEM", 3: "FP_EDEVICE", 4: "FP_ETIMEOUT", 5: "FP_EVERIFY",
             6: "FP_ERANGE"}

EXPORTED = ["vc_setup", "vc_pp_export", "vc_pp_dims", "vc_commit", "vc_commit_get", "vc_prove_all",
            "vc_proof_len", "vc_proof_get", "vc_proofs_export", "vc_proofs_state", "vc_proofs_step2_parts",
            "fp_pp_free", "fp_commit_free", "fp_proofs_free", "fp_strerror", "fp_last_error", "fp_launch_count",
            "fp_profile_enable", "fp_profile_report", "fp_profile_launches", "fp_imad_probe", "fp_fq_mul_latency", "fp_fq_mul_split_latency", "vc_commit_rows_noalloc",
            "fp_g1_bases_from_scalars", "fp_g1_bases_load", "fp_g1_bases_count", "fp_g1_bases_free", "fp_msm_g1",
            "fp_msm_window", "fp_msm_autotune", "vc_prove_one", "vc_pp_view", "vc_commit_async",
            "vc_commit_status", "vc_prove_all_batch", "vc_verify", "vc_verify_all", "vc_setup_split",
            "vc_pp_view_split", "vc_open_segments", "vc_segment_proof_len", "vc_segment_proof_get",
            "vc_verify_segment", "vc_eval_proof_len", "vc_eval_prove", "vc_eval_verify", "fp_set_schedule",
            "fp_get_schedule", "fp_batch_last_times", "fp_engine_limits_default", "fp_set_engine_limits",
            "fp_get_engine_limits", "fp_msm_window_g2"]

LIMIT_FIELDS = ["miller_block_max", "miller_warp_max", "miller_group_min", "commit_block_max", "commit_warp_max",
                "fe_block_max", "fe_warp_max", "pair_block_max", "fold_warp_max", "wterm_warp_max", "msm_chunks",
                "msm_segment_threads"]


class _Limits(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in LIMIT_FIELDS]

SCHEDULES = {"direct": 0, "lookahead": 1}


class FlexProofsError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        detail = ""
        if _lib is not None:
            detail = _lib.fp_last_error().decode(errors="replace")
        super().__init__(f"{fn}: {FP_STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    L = ctypes.CDLL(path)
    vp, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    pp = ctypes.POINTER(vp)
    L.vc_setup.argtypes = [u32, u32, u64, vp, pp]
    L.vc_pp_export.argtypes = [vp, vp, sz, ctypes.POINTER(sz)]
    L.vc_pp_dims.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
    L.vc_commit.argtypes = [vp, vp, ctypes.c_int, vp, pp]
    L.vc_commit_get.argtypes = [vp, vp, vp]
    L.vc_prove_all.argtypes = [vp, vp, u32, vp, pp]
    L.vc_proof_len.argtypes = [vp, u32, u64]
    L.vc_proof_len.restype = sz
    L.vc_proof_get.argtypes = [vp, u64, vp, sz, ctypes.POINTER(sz)]
    L.vc_prove_one.argtypes = [vp, vp, u32, u64, vp, vp, sz, ctypes.POINTER(sz)]
    L.vc_pp_view.argtypes = [vp, u32, pp]
    L.vc_verify.argtypes = [vp, vp, u32, u64, vp, vp, sz, vp]
    L.vc_verify_all.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.POINTER(u64)]
    L.vc_setup_split.argtypes = [u32, u32, u32, u64, vp, pp]
    L.vc_pp_view_split.argtypes = [vp, u32, u32, pp]
    L.vc_open_segments.argtypes = [vp, vp, u32, u32, u32, vp, pp]
    L.vc_segment_proof_len.argtypes = [vp, u32, u32]
    L.vc_segment_proof_len.restype = sz
    L.vc_segment_proof_get.argtypes = [vp, u32, vp, sz, ctypes.POINTER(sz)]
    L.vc_verify_segment.argtypes = [vp, vp, u32, u32, vp, vp, sz, vp]
    L.vc_eval_proof_len.argtypes = [vp]
    L.vc_eval_proof_len.restype = sz
    L.vc_eval_prove.argtypes = [vp, vp, vp, vp, vp, sz, ctypes.POINTER(sz)]
    L.vc_eval_verify.argtypes = [vp, vp, vp, vp, sz, vp]
    L.vc_commit_async.argtypes = [vp, vp, ctypes.c_int, vp, pp]
    L.vc_commit_status.argtypes = [vp]
    L.vc_prove_all_batch.argtypes = [u32, vp, ctypes.c_int, vp, vp]
    L.vc_proofs_export.argtypes = [vp, u64, u64, vp, sz, ctypes.POINTER(sz)]
    L.vc_proofs_state.argtypes = [vp, vp, sz, ctypes.POINTER(sz)]
    L.vc_proofs_step2_parts.argtypes = [vp, vp, vp, vp, vp]
    for n in ("fp_pp_free", "fp_commit_free", "fp_proofs_free"):
        getattr(L, n).argtypes = [vp]
        getattr(L, n).restype = None
    L.fp_strerror.argtypes = [ctypes.c_int]
    L.fp_strerror.restype = ctypes.c_char_p
    L.fp_last_error.restype = ctypes.c_char_p
    L.fp_launch_count.restype = ctypes.c_uint64
    L.fp_profile_enable.argtypes = [ctypes.c_int]
    L.fp_profile_enable.restype = None
    L.fp_profile_report.argtypes = [ctypes.c_char_p, sz]
    L.fp_profile_report.restype = sz
    L.fp_profile_launches.argtypes = [ctypes.c_char_p, sz]
    L.fp_profile_launches.restype = sz
    L.fp_imad_probe.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.fp_fq_mul_latency.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.fp_fq_mul_split_latency.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.vc_commit_rows_noalloc.argtypes = [vp, vp, vp, vp]
    L.fp_g1_bases_from_scalars.argtypes = [vp, u64, ctypes.c_int, vp, pp]
    L.fp_g1_bases_load.argtypes = [vp, u64, ctypes.c_int, vp, pp]
    L.fp_g1_bases_count.argtypes = [vp]
    L.fp_g1_bases_count.restype = u64
    L.fp_g1_bases_free.argtypes = [vp]
    L.fp_g1_bases_free.restype = None
    L.fp_msm_g1.argtypes = [vp, vp, u64, u32, ctypes.c_int, ctypes.c_int, vp, vp]
    L.fp_msm_window.argtypes = [u64, u32]
    L.fp_msm_window.restype = ctypes.c_int
    L.fp_msm_window_g2.argtypes = [u64, u32]
    L.fp_msm_window_g2.restype = ctypes.c_int
    L.fp_msm_autotune.argtypes = [vp, vp, u64, u32, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.fp_set_schedule.argtypes = [ctypes.c_int]
    L.fp_get_schedule.restype = ctypes.c_int
    L.fp_batch_last_times.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3
    for n in ("fp_engine_limits_default", "fp_set_engine_limits", "fp_get_engine_limits"):
        getattr(L, n).argtypes = [ctypes.POINTER(_Limits)]
    _lib = L
    return L


def _check(fn: str, st: int):
    if st != 0:
        raise FlexProofsError(fn, st)


def set_schedule(name: str) -> None:
    """Step-1 round schedule for later calls: "direct" (default) or "lookahead" (fp_set_schedule);
    proofs are identical under every schedule."""
    _check("fp_set_schedule", load().fp_set_schedule(SCHEDULES[name]))


def batch_last_times() -> dict:
    """Host phases (ms) of this thread's last graph-captured vc_prove_all_batch call."""
    v = [ctypes.c_double() for _ in range(3)]
    _check("fp_batch_last_times", load().fp_batch_last_times(*[ctypes.byref(x) for x in v]))
    return {"capture_ms": v[0].value, "instantiate_ms": v[1].value, "run_ms": v[2].value}


def default_engine_limits() -> dict:
    lim = _Limits()
    _check("fp_engine_limits_default", load().fp_engine_limits_default(ctypes.byref(lim)))
    return {f: getattr(lim, f) for f in LIMIT_FIELDS}


def engine_limits() -> dict:
    """The current engine-choice limits (fp_get_engine_limits)."""
    lim = _Limits()
    _check("fp_get_engine_limits", load().fp_get_engine_limits(ctypes.byref(lim)))
    return {f: getattr(lim, f) for f in LIMIT_FIELDS}


def set_engine_limits(limits: dict | None = None) -> None:
    """Set the engine-choice limits for later calls (fp_set_engine_limits): fields not given keep
    their defaults; None restores every default."""
    if limits is None:
        _check("fp_set_engine_limits", load().fp_set_engine_limits(None))
        return
    unknown = set(limits) - set(LIMIT_FIELDS)
    if unknown:
        raise ValueError(f"unknown engine limits: {sorted(unknown)}")
    vals = dict(default_engine_limits(), **limits)
    lim = _Limits(**{f: min(int(vals[f]), 0xFFFFFFFF) for f in LIMIT_FIELDS})
    _check("fp_set_engine_limits", load().fp_set_engine_limits(ctypes.byref(lim)))


def get_schedule() -> str:
    v = load().fp_get_schedule()
    return next(k for k, q in SCHEDULES.items() if q == v)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)          # torch.cuda.Stream


class PP:
    """Handle of vc_setup's device-resident public parameters (or, with parent=, a vc_pp_view of a
    larger setup for size 2^log_n).  log_r (default floor(log_n / 2)) splits N into R = 2^log_r
    segments of M = N / R elements (vc_setup_split / vc_pp_view_split)."""

    def __init__(self, log_n: int, b: int = 1, seed: int = 0, stream=None, parent: "PP | None" = None,
                 log_r: int | None = None):
        L = load()
        h = ctypes.c_void_p()
        if parent is not None:
            if log_r is None:
                _check("vc_pp_view", L.vc_pp_view(parent.h, log_n, ctypes.byref(h)))
            else:
                _check("vc_pp_view_split", L.vc_pp_view_split(parent.h, log_r, log_n - log_r, ctypes.byref(h)))
            self.parent = parent                     # keeps the parent alive while the view lives
        elif log_r is not None:
            _check("vc_setup_split", L.vc_setup_split(log_r, log_n - log_r, b, seed, _stream_ptr(stream),
                                                      ctypes.byref(h)))
        else:
            _check("vc_setup", L.vc_setup(log_n, b, seed, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        ln, R, M = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        L.vc_pp_dims(h, ctypes.byref(ln), ctypes.byref(R), ctypes.byref(M))
        self.log_n, self.R, self.M = ln.value, R.value, M.value
        self.N = self.R * self.M
        self.log_r = self.R.bit_length() - 1
        self.log_c = self.M.bit_length() - 1

    def export(self) -> bytes:
        L = load()
        n = ctypes.c_size_t()
        _check("vc_pp_export", L.vc_pp_export(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check("vc_pp_export", L.vc_pp_export(self.h, buf, n.value, ctypes.byref(n)))
        return buf.raw

    def proof_len(self, b: int, i: int) -> int:
        return load().vc_proof_len(self.h, b, i)

    def view(self, log_n: int, log_r: int | None = None) -> "PP":
        return PP(log_n, parent=self, log_r=log_r)

    def segment_proof_len(self, b: int, j: int) -> int:
        return load().vc_segment_proof_len(self.h, b, j)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.fp_pp_free(self.h)
            self.h = None


class Commitment:
    """Handle of vc_commit: C, the row commitments and the device copy of m.  With sync=False the
    commitment is only enqueued (vc_commit_async); status() then reports the range check."""

    def __init__(self, pp: PP, m, stream=None, sync: bool = True):
        L = load()
        self.pp = pp
        h = ctypes.c_void_p()
        if hasattr(m, "data_ptr"):                       # torch tensor on the device (N x 4 int64)
            assert m.is_cuda and m.is_contiguous() and m.numel() == 4 * pp.N
            ptr, on_dev = m.data_ptr(), 1
            self._keep = m
        else:
            arr = np.ascontiguousarray(m, dtype=np.uint64)
            assert arr.size == 4 * pp.N
            ptr, on_dev = arr.ctypes.data, 0
            self._keep = arr
        fn = L.vc_commit if sync else L.vc_commit_async
        _check("vc_commit", fn(pp.h, ptr, on_dev, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h

    def status(self) -> int:
        """0 if every value of m was < r, else FP_ERANGE (6); waits for this commitment's work."""
        return int(load().vc_commit_status(self.h))

    def get(self, rows: bool = True):
        C = ctypes.create_string_buffer(576)
        rb = ctypes.create_string_buffer(96 * self.pp.R) if rows else None
        _check("vc_commit_get", load().vc_commit_get(self.h, C, rb))
        return C.raw, (rb.raw if rows else None)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.fp_commit_free(self.h)
            self.h = None


class Proofs:
    """Handle of vc_prove_all's device-resident shared proof pieces."""

    def __init__(self, pp: PP, cm: Commitment, b: int, stream=None, handle=None):
        L = load()
        self.pp, self.cm, self.b = pp, cm, b
        if handle is not None:                       # from vc_prove_all_batch
            self.h = handle
            return
        h = ctypes.c_void_p()
        _check("vc_prove_all", L.vc_prove_all(pp.h, cm.h, b, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h

    def segment_proof(self, j: int) -> bytes:
        """Segment j's proof (OpenAll for sub-arrays): its block's row commitments and pi_{C_k}."""
        n = self.pp.segment_proof_len(self.b, j)
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t()
        _check("vc_segment_proof_get", load().vc_segment_proof_get(self.h, j, buf, n, ctypes.byref(ln)))
        return buf.raw[: ln.value]

    def proof(self, i: int) -> bytes:
        n = self.pp.proof_len(self.b, i)
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t()
        _check("vc_proof_get", load().vc_proof_get(self.h, i, buf, n, ctypes.byref(ln)))
        return buf.raw[: ln.value]

    def export(self, i0: int, count: int) -> bytes:
        L = load()
        ln = ctypes.c_size_t()
        _check("vc_proofs_export", L.vc_proofs_export(self.h, i0, count, None, 0, ctypes.byref(ln)))
        buf = ctypes.create_string_buffer(ln.value)
        _check("vc_proofs_export", L.vc_proofs_export(self.h, i0, count, buf, ln.value, ctypes.byref(ln)))
        return buf.raw

    def state(self) -> bytes:
        """The shared proof state as bytes (layout in include/flexproofs.h, vc_proofs_state)."""
        n = self.state_size()
        buf = ctypes.create_string_buffer(n)
        ln = ctypes.c_size_t()
        _check("vc_proofs_state", load().vc_proofs_state(self.h, buf, n, ctypes.byref(ln)))
        return buf.raw

    def state_size(self) -> int:
        ln = ctypes.c_size_t()
        _check("vc_proofs_state", load().vc_proofs_state(self.h, None, 0, ctypes.byref(ln)))
        return ln.value

    def state_into(self, host_buf) -> int:
        """Copy the shared proof state into a preallocated host buffer (numpy uint8 / pinned)."""
        ln = ctypes.c_size_t()
        ptr = host_buf.ctypes.data if hasattr(host_buf, "ctypes") else host_buf.data_ptr()
        cap = host_buf.nbytes if hasattr(host_buf, "nbytes") else host_buf.numel()
        _check("vc_proofs_state", load().vc_proofs_state(self.h, ptr, cap, ctypes.byref(ln)))
        return ln.value

    def step2_parts(self):
        R, M = self.pp.R, self.pp.M
        root, rj, gs, ds = (ctypes.create_string_buffer(n) for n in (32, 32 * R, 32 * M, 96))
        _check("vc_proofs_step2_parts", load().vc_proofs_step2_parts(self.h, root, rj, gs, ds))
        return root.raw, rj.raw, gs.raw, ds.raw

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.fp_proofs_free(self.h)
            self.h = None


# names of the C ABI, for callers who prefer them
def vc_setup(log_n: int, b: int = 1, seed: int = 0, stream=None) -> PP:
    return PP(log_n, b, seed, stream)


def vc_commit(pp: PP, m, stream=None) -> Commitment:
    return Commitment(pp, m, stream)


def vc_prove_all(pp: PP, cm: Commitment, b: int, stream=None) -> Proofs:
    return Proofs(pp, cm, b, stream)


def vc_proof_get(pf: Proofs, i: int) -> bytes:
    return pf.proof(i)


class _Job(ctypes.Structure):
    _fields_ = [("cm", ctypes.c_void_p), ("b", ctypes.c_uint32)]


def vc_prove_all_batch(jobs, use_graph: bool = False, stream=None) -> list:
    """jobs: list of (Commitment, b).  One Proofs handle per job (vc_prove_all_batch)."""
    L = load()
    n = len(jobs)
    arr = (_Job * max(1, n))(*[_Job(cm.h.value, b) for cm, b in jobs])
    outs = (ctypes.c_void_p * max(1, n))()
    _check("vc_prove_all_batch", L.vc_prove_all_batch(n, arr, int(use_graph), _stream_ptr(stream), outs))
    return [Proofs(cm.pp, cm, b, handle=ctypes.c_void_p(outs[j])) for j, (cm, b) in enumerate(jobs)]


def vc_verify(pp: PP, C: bytes, b: int, i: int, m_i: int, proof: bytes, stream=None) -> bool:
    """VC.Verify of one proof on the GPU: True if it verifies (FP_OK), False if not (FP_EVERIFY)."""
    limbs = (ctypes.c_uint64 * 4)(*[(m_i >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(4)])
    st = load().vc_verify(pp.h, C, b, i, limbs, proof, len(proof), _stream_ptr(stream))
    if st not in (0, 5):
        raise FlexProofsError("vc_verify", st)
    return st == 0


def vc_verify_all(pf: "Proofs", C: bytes, m, each: bool = False, stream=None):
    """VC.Verify of all N proofs of `pf` for the claimed values m (N x 4 uint64 limbs: numpy, or a
    torch CUDA tensor of int64) against C.  Returns (ok: numpy bool array of N, number accepted).
    each=True gives every proof its own PST check (no column sharing)."""
    N = pf.pp.N
    if hasattr(m, "data_ptr"):
        assert m.is_cuda and m.is_contiguous() and m.numel() == 4 * N
        ptr, dev, keep = m.data_ptr(), 1, m
    else:
        keep = np.ascontiguousarray(m, dtype=np.uint64)
        assert keep.size == 4 * N
        ptr, dev = keep.ctypes.data, 0
    ok = np.zeros(N, np.uint8)
    n_ok = ctypes.c_uint64()
    _check("vc_verify_all", load().vc_verify_all(pf.pp.h, C, ptr, dev, pf.h, int(each), _stream_ptr(stream),
                                                 ok.ctypes.data, ctypes.byref(n_ok)))
    del keep
    return ok.astype(bool), int(n_ok.value)


def vc_open_segments(pp: PP, cm: Commitment, b: int, k0: int = 0, nblocks: int = 0, stream=None) -> "Proofs":
    """OpenAll for sub-arrays: Step 1 only, for blocks k0 .. k0 + nblocks - 1 (0: all from k0)."""
    h = ctypes.c_void_p()
    _check("vc_open_segments", load().vc_open_segments(pp.h, cm.h, b, k0, nblocks, _stream_ptr(stream),
                                                       ctypes.byref(h)))
    return Proofs(pp, cm, b, handle=h)


def vc_verify_segment(pp: PP, C: bytes, b: int, j: int, m_j, proof: bytes, stream=None) -> bool:
    """Verifier V_j of OpenAll for sub-arrays on the GPU (m_j: M x 4 uint64 limbs)."""
    arr = np.ascontiguousarray(m_j, dtype=np.uint64)
    assert arr.size == 4 * pp.M
    st = load().vc_verify_segment(pp.h, C, b, j, arr.ctypes.data, proof, len(proof), _stream_ptr(stream))
    if st not in (0, 5):
        raise FlexProofsError("vc_verify_segment", st)
    return st == 0


def vc_eval_prove(pp: PP, cm: Commitment, r, stream=None) -> bytes:
    """Evaluation proof of the committed vector's multilinear extension at r = (r_0 .. r_{log N - 1})
    (canonical Fr integers): y || C_F || pi_FC || pi_PST."""
    assert len(r) == pp.log_n
    rb = b"".join(int(v).to_bytes(32, "big") for v in r)
    L = load()
    n = L.vc_eval_proof_len(pp.h)
    buf = ctypes.create_string_buffer(n)
    ln = ctypes.c_size_t()
    _check("vc_eval_prove", L.vc_eval_prove(pp.h, cm.h, rb, _stream_ptr(stream), buf, n, ctypes.byref(ln)))
    return buf.raw[: ln.value]


def vc_eval_verify(pp: PP, C: bytes, r, proof: bytes, stream=None) -> bool:
    """GPU verifier of vc_eval_prove's proof at r."""
    assert len(r) == pp.log_n
    rb = b"".join(int(v).to_bytes(32, "big") for v in r)
    st = load().vc_eval_verify(pp.h, C, rb, proof, len(proof), _stream_ptr(stream))
    if st not in (0, 5):
        raise FlexProofsError("vc_eval_verify", st)
    return st == 0


def vc_prove_one(pp: PP, cm: Commitment, b: int, i: int, stream=None) -> bytes:
    """pi_i alone: Step 1 on the block of i, Step 2 in full (synchronises)."""
    L = load()
    ln = ctypes.c_size_t()
    _check("vc_prove_one", L.vc_prove_one(pp.h, cm.h, b, i, _stream_ptr(stream), None, 0, ctypes.byref(ln)))
    buf = ctypes.create_string_buffer(ln.value)
    _check("vc_prove_one", L.vc_prove_one(pp.h, cm.h, b, i, _stream_ptr(stream), buf, ln.value, ctypes.byref(ln)))
    return buf.raw[: ln.value]


def launch_count() -> int:
    return int(load().fp_launch_count())


def profile_enable(on: bool = True) -> None:
    load().fp_profile_enable(int(on))


def profile_report() -> dict:
    """{kernel name: (launches, total_ms)} since the last report (synchronises)."""
    L = load()
    n = L.fp_profile_report(None, 0)
    buf = ctypes.create_string_buffer(n)
    L.fp_profile_report(buf, n)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def profile_launches() -> list:
    """[(kernel name, start_ms, ms)] per timed launch, in issue order, of the launches the last
    profile_report synchronised (start_ms from the first listed launch's start)."""
    L = load()
    n = L.fp_profile_launches(None, 0)
    buf = ctypes.create_string_buffer(n)
    L.fp_profile_launches(buf, n)
    out = []
    for line in buf.value.decode().splitlines():
        name, start, ms = line.split()
        out.append((name, float(start), float(ms)))
    return out


def imad_peak() -> float:
    """Measured 32-bit multiply-add lane operations per second of the current GPU."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check("fp_imad_probe", load().fp_imad_probe(ctypes.byref(ops), ctypes.byref(ms)))
    return ops.value


def fq_mul_latency_ns() -> float:
    """Measured latency of one dependent Fq Montgomery product on one lane (ns)."""
    ns = ctypes.c_double()
    _check("fp_fq_mul_latency", load().fp_fq_mul_latency(ctypes.byref(ns)))
    return ns.value


def fq_mul_split_latency_ns() -> float:
    """Measured latency of one dependent Fq product split over a 128-thread block's warps (ns)."""
    ns = ctypes.c_double()
    _check("fp_fq_mul_split_latency", load().fp_fq_mul_split_latency(ctypes.byref(ns)))
    return ns.value


def vc_commit_rows_noalloc(pp: PP, m_dev, rows_dev, stream=None) -> None:
    """Row commitments into a caller-provided device buffer, without device allocation
    (see include/flexproofs.h).  m_dev / rows_dev: device tensors (N x 4 int64, R*96 uint8)."""
    _check("vc_commit_rows_noalloc",
           load().vc_commit_rows_noalloc(pp.h, m_dev.data_ptr(), rows_dev.data_ptr(), _stream_ptr(stream)))


def _ptr_of(x):
    """(pointer, on_device, keep-alive) of a torch CUDA tensor, numpy array or bytes."""
    if hasattr(x, "data_ptr"):
        assert x.is_cuda and x.is_contiguous()
        return x.data_ptr(), 1, x
    if isinstance(x, (bytes, bytearray)):
        arr = np.frombuffer(bytes(x), dtype=np.uint8)
        return arr.ctypes.data, 0, arr
    arr = np.ascontiguousarray(x)
    return arr.ctypes.data, 0, arr


class G1Bases:
    """Device-resident bases of fp_msm_g1: from scalars (P_i = s_i g1; n x 4 uint64 limbs) or from
    serialised affine points (n x 96 bytes)."""

    def __init__(self, scalars=None, points=None, stream=None):
        L = load()
        h = ctypes.c_void_p()
        if scalars is not None:
            ptr, dev, keep = _ptr_of(scalars if hasattr(scalars, "data_ptr") else
                                     np.ascontiguousarray(scalars, dtype=np.uint64))
            n = (scalars.numel() if hasattr(scalars, "numel") else keep.size) // 4
            _check("fp_g1_bases_from_scalars", L.fp_g1_bases_from_scalars(ptr, n, dev, _stream_ptr(stream),
                                                                          ctypes.byref(h)))
        else:
            ptr, dev, keep = _ptr_of(points)
            n = (points.numel() if hasattr(points, "numel") else keep.size) // 96
            _check("fp_g1_bases_load", L.fp_g1_bases_load(ptr, n, dev, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.n = int(L.fp_g1_bases_count(h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.fp_g1_bases_free(self.h)
            self.h = None


def msm_g1(bases: G1Bases, k, nbatch: int = 1, window: int = 0, stream=None, out=None):
    """sum_i k[j n + i] P[(j n + i) mod npts] for j < nbatch.  Host input (numpy n*nbatch x 4
    uint64): returns nbatch x 96 bytes.  Device input (torch int64 tensor): enqueues into the
    device uint8 tensor `out` (nbatch * 96) and returns it."""
    L = load()
    if hasattr(k, "data_ptr"):
        n = k.numel() // 4 // nbatch
        assert out is not None and out.is_cuda and out.numel() >= 96 * nbatch
        _check("fp_msm_g1", L.fp_msm_g1(bases.h, k.data_ptr(), n, nbatch, 1, window, _stream_ptr(stream),
                                        out.data_ptr()))
        return out
    arr = np.ascontiguousarray(k, dtype=np.uint64)
    n = arr.size // 4 // nbatch
    buf = ctypes.create_string_buffer(96 * nbatch)
    _check("fp_msm_g1", L.fp_msm_g1(bases.h, arr.ctypes.data if arr.size else None, n, nbatch, 0, window,
                                    _stream_ptr(stream), buf))
    return buf.raw


def msm_window(n: int, nbatch: int = 1) -> int:
    return int(load().fp_msm_window(n, nbatch))


def msm_window_g2(n: int, nbatch: int = 1) -> int:
    return int(load().fp_msm_window_g2(n, nbatch))


def msm_autotune(bases: G1Bases, k_dev, nbatch: int = 1, stream=None):
    """Measured best window for this shape (kept for later calls with window 0) and its time in ms."""
    c, ms = ctypes.c_int(), ctypes.c_double()
    n = k_dev.numel() // 4 // nbatch
    _check("fp_msm_autotune", load().fp_msm_autotune(bases.h, k_dev.data_ptr(), n, nbatch, _stream_ptr(stream),
                                                     ctypes.byref(c), ctypes.byref(ms)))
    return c.value, ms.value
