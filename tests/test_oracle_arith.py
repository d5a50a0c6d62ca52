"""Pins of the oracle's arithmetic layer against things other than itself: Python integers,
hashlib, the curve order, brute force and closed forms (BLS12-381, x = -0xd201000000010000)."""
import hashlib
import os
import random

import pytest

import oracle as O
from tests import _pyref as ref

rng = random.Random(1234)


def test_constants_derived_from_x():
    assert O.const_p() == ref.P
    assert O.const_r() == ref.R
    assert ref.P.bit_length() == 381 and ref.R.bit_length() == 255
    # the final exponent is exactly (p^12 - 1) / r and r divides p^12 - 1
    assert (ref.P**12 - 1) % ref.R == 0
    assert O.const_final_exp() == (ref.P**12 - 1) // ref.R
    assert O.const_final_exp().bit_length() == 4314
    # #E(Fq) = p - x = h1 r with h1 = (x-1)^2/3
    assert ref.P - ref.X == ((ref.X - 1) ** 2 // 3) * ref.R


@pytest.mark.parametrize("op", ["add", "sub", "mul", "inv"])
def test_fq_ops_vs_python(op):
    for _ in range(50):
        a, b = rng.randrange(ref.P), rng.randrange(ref.P)
        exp = {"add": (a + b) % ref.P, "sub": (a - b) % ref.P, "mul": a * b % ref.P,
               "inv": pow(a, -1, ref.P) if a else 0}[op]
        assert O.fq_op(op, a, b) == exp
    # edges
    assert O.fq_op("mul", ref.P - 1, ref.P - 1) == 1
    assert O.fq_op("add", ref.P - 1, 1) == 0
    assert O.fq_op("inv", 0) == 0


@pytest.mark.parametrize("op", ["add", "sub", "mul", "inv"])
def test_fr_ops_vs_python(op):
    for _ in range(50):
        a, b = rng.randrange(ref.R), rng.randrange(ref.R)
        exp = {"add": (a + b) % ref.R, "sub": (a - b) % ref.R, "mul": a * b % ref.R,
               "inv": pow(a, -1, ref.R) if a else 0}[op]
        assert O.fr_op(op, a, b) == exp


def test_fermat_and_inverse_identities():
    for _ in range(5):
        a = rng.randrange(1, ref.P)
        assert O.fq_op("mul", a, O.fq_op("inv", a)) == 1


def test_fq2_mul_vs_python():
    for _ in range(20):
        a = (rng.randrange(ref.P), rng.randrange(ref.P))
        b = (rng.randrange(ref.P), rng.randrange(ref.P))
        exp = ((a[0] * b[0] - a[1] * b[1]) % ref.P, (a[0] * b[1] + a[1] * b[0]) % ref.P)
        assert O.fq2_mul(a, b) == exp


def test_wide_reduction_vs_python():
    for n in (1, 31, 32, 33, 64):
        d = os.urandom(n)
        assert O.fr_from_wide(d) == int.from_bytes(d, "big") % ref.R


@pytest.mark.parametrize("n", [0, 1, 3, 55, 56, 57, 63, 64, 65, 119, 120, 128, 1000])
def test_sha256_vs_hashlib(n):
    m = os.urandom(n)
    assert O.sha256(m) == hashlib.sha256(m).digest()


def test_hfr_vs_python():
    for tag in ("FP-r", "FP-x", "FP-rho"):
        for n in (0, 5, 36, 200):
            d = os.urandom(n)
            assert O.hfr(tag, d) == ref.hfr(tag, d)


def test_splitmix_matches_published_definition():
    # SplitMix64: state += gamma; z = mix(state); Fr by rejection with top limb masked
    def sm(seed):
        s = seed
        while True:
            s = (s + 0x9E3779B97F4A7C15) % 2**64
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % 2**64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % 2**64
            yield z ^ (z >> 31)
    g = sm(42)
    exp = []
    while len(exp) < 50:
        w = [next(g) for _ in range(4)]
        v = w[0] | (w[1] << 64) | (w[2] << 128) | ((w[3] & (2**63 - 1)) << 192)
        if v < ref.R:
            exp.append(v)
    assert O.splitmix_fr(42, 50) == exp
    from paper_2601_03031_gb300 import inputs
    assert inputs.to_ints(inputs.fr_uniform(42, 50)) == exp


def test_generators_on_curve_and_order_r():
    g1, g2 = O.g1_gen(), O.g2_gen()
    assert O.g1_valid(g1) and O.g2_valid(g2)
    assert O.g1_mul(g1, ref.R) == bytes(96)
    assert O.g2_mul(g2, ref.R) == bytes(192)
    assert O.g1_mul(g1, ref.R - 1) != bytes(96)
    # the G1 affine coordinates satisfy y^2 = x^3 + 4 in Python integers
    x, y = int.from_bytes(g1[:48], "big"), int.from_bytes(g1[48:], "big")
    assert (y * y - x**3 - 4) % ref.P == 0


def test_group_law_brute_force():
    g1, g2 = O.g1_gen(), O.g2_gen()
    acc1, acc2 = bytes(96), bytes(192)
    for k in range(1, 12):
        acc1 = O.g1_add(acc1, g1)
        acc2 = O.g2_add(acc2, g2)
        assert O.g1_mul(g1, k) == acc1
        assert O.g2_mul(g2, k) == acc2
    assert O.g1_dbl(g1) == O.g1_mul(g1, 2)
    assert O.g1_add(g1, O.g1_mul(g1, ref.R - 1)) == bytes(96)
    a, b = rng.randrange(ref.R), rng.randrange(ref.R)
    assert O.g1_add(O.g1_mul(g1, a), O.g1_mul(g1, b)) == O.g1_mul(g1, (a + b) % ref.R)
    assert O.g2_add(O.g2_mul(g2, a), O.g2_mul(g2, b)) == O.g2_mul(g2, (a + b) % ref.R)
    assert O.g1_mul(O.g1_mul(g1, a), b) == O.g1_mul(g1, a * b % ref.R)


def test_msm_closed_form():
    # P_i = s_i g1 with known s_i, so sum k_i P_i = (sum k_i s_i mod r) g1
    g1 = O.g1_gen()
    s = [rng.randrange(ref.R) for _ in range(6)]
    k = [rng.randrange(2**255) for _ in range(6)]
    pts = b"".join(O.g1_mul(g1, v) for v in s)
    assert O.g1_msm(pts, k) == O.g1_mul(g1, sum(a * b for a, b in zip(k, s)) % ref.R)
