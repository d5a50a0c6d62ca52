"""The lane-parallel device engines, compiled for the host and checked against the oracle (no GPU).

`tests/emu/engines.cpp` includes the CUDA engine headers (warp12.cuh, group_ec.cuh) through a shim
(`tests/emu/lane_shim.h`) that runs every lane of a warp or block as a host thread, with the
warp/block barriers as one barrier over all of them and the PTX carry-chain primitives in 64-bit
host arithmetic.  The same source the GPU runs is thus checked on the CPU, exactly:
- the Miller loop on a warp and on a 128-thread block: its final exponentiation (by the oracle)
  equals the oracle's pairing (line scalings vanish under it, so the Miller values themselves may
  differ);
- the final exponentiation on a warp and on a block against the oracle's plain square-and-multiply
  by (p^12 - 1)/r;
- exponentiation in GT by the Frobenius split of the exponent (gt_exp.cuh), whole and in parts,
  against the oracle's square-and-multiply;
- G1 scalar multiplication on an 8-lane group (GLV, 2-bit joint windows) and G2 on a warp (GLS),
  whole and split in 2 and 4 parts on shifted bases 2^(128 p / NP) P and 2^(64 p / NP) Q formed by
  the engines' own doublings (Step 1's split folds), against the oracle's double-and-add, for edge
  and random scalars and the identity.
"""
import ctypes
import os
import random
import shutil
import subprocess

import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_03031_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    lib = str(tmp_path_factory.mktemp("emu") / "libengines.so")
    subprocess.check_call([gxx, "-std=c++20", "-O1", "-shared", "-fPIC", f"-I{CSRC}", "-o", lib,
                           os.path.join(HERE, "emu", "engines.cpp")])
    L = ctypes.CDLL(lib)
    for n in ("emu_fq_mul_split", "emu_miller", "emu_final_exp", "emu_gt_pow", "emu_g1_mul", "emu_g1_dbl_n", "emu_g2_mul",
              "emu_g2_dbl_n", "emu_g1_comb", "emu_g2_comb"):
        getattr(L, n).restype = None
    return L


R = O.const_r()


def words(k: int):
    return (ctypes.c_uint32 * 8)(*[(k >> (32 * i)) & 0xFFFFFFFF for i in range(8)])


def g1_mul(L, P, k, np_=1, part=0):
    o = ctypes.create_string_buffer(96)
    L.emu_g1_mul(P, words(k), np_, part, o)
    return o.raw


def g2_mul(L, Q, k, np_=1, part=0):
    o = ctypes.create_string_buffer(192)
    L.emu_g2_mul(Q, words(k), np_, part, o)
    return o.raw


def test_fq_product_split_over_four_warps(emu):
    """fq_split.cuh: every warp's lane t ends with x_t y_t 2^-384 mod p, canonical, for random operands
    and the edges 0, 1, p - 1, p - 2, 2^380, 2^381 - 1 mod p (the largest T and S the bounds allow)."""
    P = O.const_p()
    rnd = random.Random(23)
    edges = [0, 1, P - 1, P - 2, 1 << 380, ((1 << 381) - 1) % P, (1 << 32) - 1, 1 << 352]
    pairs = [(a, b) for a in edges for b in (P - 1, edges[-3], 1)]
    pairs += [(rnd.randrange(P), rnd.randrange(P)) for _ in range(96 - len(pairs))]
    rinv = pow(1 << 384, -1, P)
    for i in range(0, len(pairs), 32):
        batch = pairs[i:i + 32]
        batch += [(0, 0)] * (32 - len(batch))
        xs = (ctypes.c_uint32 * 384)(*[(a >> (32 * j)) & 0xFFFFFFFF for a, _ in batch for j in range(12)])
        ys = (ctypes.c_uint32 * 384)(*[(b >> (32 * j)) & 0xFFFFFFFF for _, b in batch for j in range(12)])
        out = (ctypes.c_uint32 * (128 * 12))()
        emu.emu_fq_mul_split(xs, ys, out)
        for L in range(128):
            a, b = batch[L & 31]
            got = sum(out[12 * L + j] << (32 * j) for j in range(12))
            assert got == a * b * rinv % P, (L, hex(a), hex(b))


@pytest.mark.parametrize("nw", [1, 4])
def test_miller_loop_then_final_exp_is_the_pairing(emu, nw):
    rnd = random.Random(nw)
    for _ in range(2):
        P = O.g1_mul(O.g1_gen(), rnd.randrange(1, R))
        Q = O.g2_mul(O.g2_gen(), rnd.randrange(1, R))
        f = ctypes.create_string_buffer(576)
        emu.emu_miller(nw, P, Q, f)
        assert O.final_exp(f.raw) == O.pairing(P, Q)


@pytest.mark.parametrize("nw", [1, 4])
def test_final_exp(emu, nw):
    rnd = random.Random(10 + nw)
    for _ in range(2):
        f = O.miller(O.g1_mul(O.g1_gen(), rnd.randrange(1, R)), O.g2_mul(O.g2_gen(), rnd.randrange(1, R)))
        o = ctypes.create_string_buffer(576)
        emu.emu_final_exp(nw, f, o)
        assert o.raw == O.final_exp(f)


@pytest.mark.parametrize("nw", [1, 4])
def test_gt_exponentiation_by_frobenius_split(emu, nw):
    """g^c by the base-|x| digits of c on the Frobenius powers of g, whole and in 4 parts of 16 digit
    bits on the bases g^(2^(16 p)), against the oracle's square-and-multiply."""
    rnd = random.Random(30 + nw)
    g = O.pairing(O.g1_mul(O.g1_gen(), rnd.randrange(1, R)), O.g2_mul(O.g2_gen(), rnd.randrange(1, R)))
    for c in (0, 1, R - 1, rnd.randrange(R)):
        o = ctypes.create_string_buffer(576)
        emu.emu_gt_pow(nw, g, words(c), 0, 64, o)
        assert o.raw == O.fq12_pow(g, c), c
    c = rnd.randrange(R)
    acc = O.fq12_pow(g, 0)
    for part in range(4):
        o = ctypes.create_string_buffer(576)
        emu.emu_gt_pow(nw, O.fq12_pow(g, 1 << (16 * part)), words(c), 16 * part, 16, o)
        acc = O.fq12_mul(acc, o.raw)
    assert acc == O.fq12_pow(g, c)


def test_g1_scalar_mul_whole_and_split(emu):
    rnd = random.Random(21)
    P = O.g1_mul(O.g1_gen(), rnd.randrange(1, R))
    for k in (0, 1, 2, R - 1, rnd.randrange(R), rnd.randrange(R)):
        e = O.g1_mul(P, k)
        assert g1_mul(emu, P, k) == e, k
        for np_ in (2, 4):
            acc, base = bytes(96), P
            for part in range(np_):
                if part:
                    o = ctypes.create_string_buffer(96)
                    emu.emu_g1_dbl_n(base, 128 // np_, o)
                    base = o.raw
                    assert base == O.g1_mul(P, 1 << (128 * part // np_))
                acc = O.g1_add(acc, g1_mul(emu, base, k, np_, part))
            assert acc == e, (k, np_)
    assert g1_mul(emu, bytes(96), rnd.randrange(R), 4, 1) == bytes(96)


def test_g2_scalar_mul_whole_and_split(emu):
    rnd = random.Random(22)
    Q = O.g2_mul(O.g2_gen(), rnd.randrange(1, R))
    for k in (0, 1, 2, R - 1, rnd.randrange(R), rnd.randrange(R)):
        e = O.g2_mul(Q, k)
        assert g2_mul(emu, Q, k) == e, k
        for np_ in (2, 4):
            acc, base = bytes(192), Q
            for part in range(np_):
                if part:
                    o = ctypes.create_string_buffer(192)
                    emu.emu_g2_dbl_n(base, 64 // np_, o)
                    base = o.raw
                    assert base == O.g2_mul(Q, 1 << (64 * part // np_))
                acc = O.g2_add(acc, g2_mul(emu, base, k, np_, part))
            assert acc == e, (k, np_)
    assert g2_mul(emu, bytes(192), rnd.randrange(R), 2, 1) == bytes(192)


def test_fixed_base_combs(emu):
    """Step 1's comb folds (group_ec.cuh, k_step1.cu): the chain of doublings, the window tables of
    G1 (GLV, 2-bit windows, entries a B - b phi(B)) and the position tables of G2 (GLS, entries
    sum (-1)^j psi^j(B)), and the sum of one entry per window give k P and k Q as the oracle's
    double-and-add does, for edge and random scalars and the identity."""
    rnd = random.Random(41)
    P = O.g1_mul(O.g1_gen(), rnd.randrange(1, R))
    Q = O.g2_mul(O.g2_gen(), rnd.randrange(1, R))
    scalars = [0, 1, 2, R - 1, (1 << 128) - 1, rnd.randrange(R), rnd.randrange(R)]
    for k in scalars:
        o = ctypes.create_string_buffer(96)
        emu.emu_g1_comb(P, words(k), o)
        assert o.raw == O.g1_mul(P, k), hex(k)
    for k in scalars[:5]:
        o = ctypes.create_string_buffer(192)
        emu.emu_g2_comb(Q, words(k), o)
        assert o.raw == O.g2_mul(Q, k), hex(k)
    o = ctypes.create_string_buffer(96)
    emu.emu_g1_comb(O.g1_mul(O.g1_gen(), 0), words(5), o)
    assert o.raw == O.g1_mul(O.g1_gen(), 0)
