"""The streaming SHA-256 of the CUDA path (sha256.cuh), compiled for the host and checked against
hashlib (no GPU): messages of many lengths fed in pieces at word-aligned and unaligned cut points,
so that whole blocks hashed in place, word moves into the buffer and byte moves all run."""
import ctypes
import hashlib
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_03031_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    so = str(tmp_path_factory.mktemp("emu_sha") / "libsha.so")
    subprocess.check_call([gxx, "-std=c++20", "-O1", "-shared", "-fPIC", f"-I{CSRC}", "-o", so,
                           os.path.join(HERE, "emu", "sha.cpp")])
    L = ctypes.CDLL(so)
    L.emu_sha256_pieces.restype = None
    return L


def digest(lib, msg: bytes, cuts) -> bytes:
    buf = ctypes.create_string_buffer(msg, len(msg) + 1)     # 16-byte aligned base
    c = (ctypes.c_uint32 * max(1, len(cuts)))(*cuts)
    out = ctypes.create_string_buffer(32)
    lib.emu_sha256_pieces(buf, len(msg), c, len(cuts), out)
    return out.raw


def test_sha256_pieces_against_hashlib(lib):
    rnd = random.Random(5)
    for n in [0, 1, 3, 4, 55, 56, 63, 64, 65, 100, 128, 588, 600, 25164]:
        msg = bytes(rnd.randrange(256) for _ in range(n))
        want = hashlib.sha256(msg).digest()
        assert digest(lib, msg, []) == want
        # a statement: 576 + 12 bytes of header, then rows of 96 bytes (word moves after the header)
        for cuts in ([576, 588], [12], [5], [4, 8, 68], sorted(rnd.sample(range(n + 1), min(n, 6)))):
            cuts = [c for c in cuts if c <= n]
            assert digest(lib, msg, cuts) == want, (n, cuts)
