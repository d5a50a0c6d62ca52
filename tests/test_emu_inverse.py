"""The field inverse of the CUDA path (batched division steps, `mp::inv_ds` in fp.cuh, and its form
on the four lanes of a quad, `mp::inv_ds_quad`), compiled for the host and checked against Python's
modular inverse: x x^-1 = 1 for random and edge values of Fq and Fr (1, 2, p - 1, values with long
runs of zero or one bits), and 0 maps to 0 (no GPU)."""
import ctypes
import os
import random
import shutil
import subprocess

import pytest

from tests import _pyref as ref

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_03031_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    so = str(tmp_path_factory.mktemp("emu_inv") / "libinv.so")
    subprocess.check_call([gxx, "-std=c++20", "-O1", "-shared", "-fPIC", f"-I{CSRC}", "-o", so,
                           os.path.join(HERE, "emu", "inverse.cpp")])
    L = ctypes.CDLL(so)
    for f in (L.emu_inv_fq, L.emu_inv_fr, L.emu_inv_fq_quad, L.emu_inv_fr_quad, L.emu_inv_fq_warp):
        f.restype = None
    return L


def call(fn, x: int, n: int) -> int:
    xi = (ctypes.c_uint32 * n)(*[(x >> (32 * i)) & 0xFFFFFFFF for i in range(n)])
    r = (ctypes.c_uint32 * n)()
    fn(xi, r)
    return sum(r[i] << (32 * i) for i in range(n))


def edge_values(m: int):
    vals = [1, 2, 3, m - 1, m - 2, (m - 1) // 2, 1 << 31, (1 << 64) - 1, m >> 1, (m >> 3) | 1]
    vals += [((1 << k) - 1) % m for k in (30, 31, 32, 33, 63, 64, 200)]
    return [v % m for v in vals if v % m]


@pytest.mark.parametrize("field", ["fq", "fr"])
def test_inverse_against_python(lib, field):
    m, n, fn = (ref.P, 12, lib.emu_inv_fq) if field == "fq" else (ref.R, 8, lib.emu_inv_fr)
    rnd = random.Random(17)
    values = edge_values(m) + [rnd.randrange(1, m) for _ in range(400)]
    for x in values:
        assert call(fn, x, n) == pow(x, -1, m), hex(x)
    assert call(fn, 0, n) == 0


@pytest.mark.parametrize("field", ["fq", "fr"])
def test_quad_inverse_against_python(lib, field):
    """The quad form: the four lanes start from different values (only the first lane's is the
    input), every lane must return the first lane's inverse."""
    m, n, fn = (ref.P, 12, lib.emu_inv_fq_quad) if field == "fq" else (ref.R, 8, lib.emu_inv_fr_quad)
    rnd = random.Random(23)
    values = edge_values(m) + [rnd.randrange(1, m) for _ in range(150)] + [0]
    for x in values:
        lanes = [x] + [rnd.randrange(0, m) for _ in range(3)]
        xi = (ctypes.c_uint32 * (4 * n))(*[(v >> (32 * i)) & 0xFFFFFFFF for v in lanes for i in range(n)])
        r = (ctypes.c_uint32 * (4 * n))()
        fn(xi, r)
        want = pow(x, -1, m) if x else 0
        for q in range(4):
            got = sum(r[q * n + i] << (32 * i) for i in range(n))
            assert got == want, (hex(x), q)


def test_quad_inverse_eight_quads_of_a_warp(lib):
    """Eight quads of one warp invert eight different values at once (zero among them): each quad's
    lanes return its first lane's inverse, whatever the other quads do."""
    rnd = random.Random(29)
    n, m = 12, ref.P
    for trial in range(6):
        firsts = [rnd.randrange(1, m) for _ in range(8)]
        if trial == 0:
            firsts[3] = 0
        lanes = [firsts[q // 4] if q % 4 == 0 else rnd.randrange(0, m) for q in range(32)]
        xi = (ctypes.c_uint32 * (32 * n))(*[(v >> (32 * i)) & 0xFFFFFFFF for v in lanes for i in range(n)])
        r = (ctypes.c_uint32 * (32 * n))()
        lib.emu_inv_fq_warp(xi, r)
        for q in range(32):
            x = firsts[q // 4]
            got = sum(r[q * n + i] << (32 * i) for i in range(n))
            assert got == (pow(x, -1, m) if x else 0), (trial, q)
