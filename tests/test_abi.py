"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and exports every entry
point that include/flexproofs.h declares.  No compute calls (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flexproofs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:vc|fp)_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("vc_setup", "vc_commit", "vc_prove_all", "vc_proof_get", "fp_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2601_03031_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2601_03031_gb300 import _lib
    assert sorted(_lib.EXPORTED) == declared_functions()


def test_invalid_arguments_rejected_without_device_work():
    from paper_2601_03031_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    lib.vc_setup.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.vc_setup(1, 1, 0, None, ctypes.byref(out)) == 1       # log_n < 2
    assert lib.vc_setup(27, 1, 0, None, ctypes.byref(out)) == 1      # log_n > 26
    assert lib.vc_setup(10, 33, 0, None, ctypes.byref(out)) == 1     # b > R = 32
    assert lib.vc_setup(10, 0, 0, None, ctypes.byref(out)) == 1      # b < 1
    lib.fp_strerror.restype = ctypes.c_char_p
    assert lib.fp_strerror(6) == b"scalar out of range (>= r)"


def test_msm_window_model_and_argument_checks():
    """fp_msm_window is host logic (cost model); fp_msm_g1 rejects bad arguments before device work."""
    from paper_2601_03031_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    lib.fp_msm_window.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    ws = [lib.fp_msm_window(1 << k, 1) for k in range(8, 25)]
    assert all(4 <= w <= 16 for w in ws)
    assert ws == sorted(ws)                           # more terms never pick a smaller window
    assert lib.fp_msm_window(1024, 1024) <= lib.fp_msm_window(1 << 20, 1)
    lib.fp_msm_g1.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    buf = ctypes.create_string_buffer(96)
    assert lib.fp_msm_g1(None, None, 0, 1, 0, 0, None, buf) == 1      # no bases
    lib.fp_g1_bases_from_scalars.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.fp_g1_bases_from_scalars(None, 5, 0, None, ctypes.byref(out)) == 1   # NULL scalars, n > 0
    assert lib.fp_g1_bases_from_scalars(None, 1 << 30, 0, None, ctypes.byref(out)) == 1


def test_new_entry_points_reject_bad_arguments_without_device_work():
    """The segment, evaluation and batch-verification entry points check their arguments on the host
    (null handles, out-of-range splits) before any CUDA call."""
    from paper_2601_03031_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    out = ctypes.c_void_p()
    lib.vc_setup_split.argtypes = [u32, u32, u32, u64, vp, vp]
    assert lib.vc_setup_split(0, 4, 1, 0, None, ctypes.byref(out)) == 1      # log_r < 1
    assert lib.vc_setup_split(4, 0, 1, 0, None, ctypes.byref(out)) == 1      # log_c < 1
    assert lib.vc_setup_split(14, 4, 1, 0, None, ctypes.byref(out)) == 1     # log_r > 13
    assert lib.vc_setup_split(13, 14, 1, 0, None, ctypes.byref(out)) == 1    # N > 2^26
    assert lib.vc_setup_split(3, 3, 9, 0, None, ctypes.byref(out)) == 1      # b > R
    lib.vc_pp_view_split.argtypes = [vp, u32, u32, vp]
    assert lib.vc_pp_view_split(None, 2, 2, ctypes.byref(out)) == 1
    lib.vc_open_segments.argtypes = [vp, vp, u32, u32, u32, vp, vp]
    assert lib.vc_open_segments(None, None, 1, 0, 0, None, ctypes.byref(out)) == 1
    lib.vc_segment_proof_len.argtypes = [vp, u32, u32]
    lib.vc_segment_proof_len.restype = ctypes.c_size_t
    assert lib.vc_segment_proof_len(None, 1, 0) == 0
    lib.vc_segment_proof_get.argtypes = [vp, u32, vp, ctypes.c_size_t, vp]
    ln = ctypes.c_size_t()
    assert lib.vc_segment_proof_get(None, 0, None, 0, ctypes.byref(ln)) == 1
    lib.vc_verify_segment.argtypes = [vp, vp, u32, u32, vp, vp, ctypes.c_size_t, vp]
    assert lib.vc_verify_segment(None, None, 1, 0, None, None, 0, None) == 1
    lib.vc_eval_proof_len.argtypes = [vp]
    lib.vc_eval_proof_len.restype = ctypes.c_size_t
    assert lib.vc_eval_proof_len(None) == 0
    lib.vc_eval_prove.argtypes = [vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    assert lib.vc_eval_prove(None, None, None, None, None, 0, ctypes.byref(ln)) == 1
    lib.vc_eval_verify.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
    assert lib.vc_eval_verify(None, None, None, None, 0, None) == 1
    lib.vc_verify_all.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
    assert lib.vc_verify_all(None, None, None, 0, None, 0, None, None, None) == 1


def test_engine_limits_and_schedule_settings_on_the_host():
    """The process-wide settings need no device: defaults, partial updates, invalid values refused."""
    from paper_2601_03031_gb300 import build as B
    B.build()
    from paper_2601_03031_gb300 import _lib as F
    d = F.default_engine_limits()
    assert d["miller_block_max"] == 1024 and d["fe_block_max"] == 256 and d["msm_chunks"] == 1 << 17
    try:
        F.set_engine_limits({"fe_block_max": 0, "fold_warp_max": 7})
        cur = F.engine_limits()
        assert cur["fe_block_max"] == 0 and cur["fold_warp_max"] == 7 and cur["miller_block_max"] == 1024
        with pytest.raises(F.FlexProofsError):
            F.set_engine_limits({"msm_chunks": 0})
        with pytest.raises(ValueError):
            F.set_engine_limits({"no_such_limit": 1})
        F.set_engine_limits(None)
        assert F.engine_limits() == d
        assert F.get_schedule() == "direct"
        F.set_schedule("lookahead")
        assert F.get_schedule() == "lookahead"
        assert F.load().fp_set_schedule(7) == 1
    finally:
        F.set_engine_limits(None)
        F.set_schedule("direct")
