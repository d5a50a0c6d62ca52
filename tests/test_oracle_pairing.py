"""Pins of the oracle's pairing: bilinearity, non-degeneracy, order r, identity handling,
and equality with an independent pure-Python Miller function computed from the definition."""
import random

import pytest

import oracle as O
from tests import _pyref as ref

rng = random.Random(99)
ONE = None


def gt_one():
    return O.final_exp(O.miller(bytes(96), O.g2_gen()))   # e(O, Q) = 1


def test_bilinearity_and_nondegeneracy():
    g1, g2 = O.g1_gen(), O.g2_gen()
    e = O.pairing(g1, g2)
    assert e != gt_one()                                   # non-degenerate
    assert O.fq12_pow(e, ref.R) == gt_one()                # order r
    a, b = rng.randrange(1, ref.R), rng.randrange(1, ref.R)
    assert O.pairing(O.g1_mul(g1, a), O.g2_mul(g2, b)) == O.fq12_pow(e, a * b % ref.R)
    # e(P1 + P2, Q) = e(P1, Q) e(P2, Q)
    P1, P2 = O.g1_mul(g1, 3), O.g1_mul(g1, 11)
    assert O.pairing(O.g1_add(P1, P2), g2) == O.fq12_mul(O.pairing(P1, g2), O.pairing(P2, g2))
    Q1, Q2 = O.g2_mul(g2, 5), O.g2_mul(g2, 9)
    assert O.pairing(g1, O.g2_add(Q1, Q2)) == O.fq12_mul(O.pairing(g1, Q1), O.pairing(g1, Q2))


def test_identity_inputs_give_one():
    assert O.pairing(bytes(96), O.g2_gen()) == gt_one()
    assert O.pairing(O.g1_gen(), bytes(192)) == gt_one()
    one = gt_one()
    assert one == b"\0" * 47 + b"\1" + b"\0" * 528


def test_inverse_and_conjugation():
    g1, g2 = O.g1_gen(), O.g2_gen()
    e = O.pairing(g1, g2)
    e_neg = O.pairing(O.g1_mul(g1, ref.R - 1), g2)
    assert O.fq12_mul(e, e_neg) == gt_one()
    assert O.fq12_conj(e) == e_neg                         # unitary: inverse is the conjugate


@pytest.mark.slow
def test_pairing_equals_definition_in_pure_python():
    from tests import _pypairing
    for a, b in [(1, 1), (rng.randrange(1, ref.R), rng.randrange(1, ref.R))]:
        P = O.g1_mul(O.g1_gen(), a)
        Q = O.g2_mul(O.g2_gen(), b)
        assert O.pairing(P, Q) == _pypairing.pairing_bytes(P, Q)
