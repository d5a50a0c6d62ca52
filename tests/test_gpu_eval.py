"""Evaluation proof at a point (Sec. 4.4, "Compatibility with a family of zkSNARKs") on the GPU
against the oracle: proof bytes equal for several splits and points (the FC part runs through the
Step-1 round chain with a dense b), y at Boolean points equals the element, the oracle's and the
GPU verifier accept it and agree on every tampered part, and out-of-range coordinates are rejected."""
import random

import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402


def point(seed, n):
    rnd = random.Random(seed)
    return [rnd.randrange(I.R_INT) for _ in range(n)]


@pytest.mark.parametrize("log_n,log_r", [(4, 2), (5, 2), (7, 3), (6, 5), (8, 1), (10, 5)])
def test_eval_proof_equals_oracle(log_n, log_r, schedule):
    seed = 71 + log_n
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    opp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    for ps in (1, 2):
        r = point(seed * 10 + ps, log_n)
        got = F.vc_eval_prove(pp, cm, r)
        assert got == O.eval_prove(opp, m.tobytes(), C, rows, r)
        assert O.eval_verify(opp, C, r, got)
        assert F.vc_eval_verify(pp, C, r, got)


def test_eval_boolean_points_and_range():
    log_n, seed = 6, 81
    pp = F.PP(log_n, 1, seed)
    m = I.vector(seed + 1, log_n)
    vals = I.to_ints(m)
    cm = F.Commitment(pp, m)
    for i in (0, 9, 63):
        r = [(i >> k) & 1 for k in range(log_n)]
        assert int.from_bytes(F.vc_eval_prove(pp, cm, r)[:32], "big") == vals[i]
    bad = point(5, log_n)
    bad[2] = I.R_INT
    with pytest.raises(F.FlexProofsError) as e:
        F.vc_eval_prove(pp, cm, bad)
    assert e.value.status == 6


def test_eval_n16(schedule):
    log_n, seed = 16, 0
    pp = F.PP(log_n, 1, seed)
    opp = O.PP(log_n, seed)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    beta, tau = opp.trapdoor()
    C, rows = _pyec.commit_closed_form(_pyec.Groups(O.g1_gen(), O.g2_gen()), beta, tau, opp.R, opp.M,
                                       I.to_ints(m))
    assert cm.get() == (C, rows)
    r = point(123, log_n)
    got = F.vc_eval_prove(pp, cm, r)
    assert O.eval_verify(opp, C, r, got)
    # y against the multilinear extension evaluated by folding the vector on the host
    vals = I.to_ints(m)
    cur = vals
    for k in range(log_n):
        cur = [(cur[2 * c] + r[k] * (cur[2 * c + 1] - cur[2 * c])) % I.R_INT for c in range(len(cur) // 2)]
    assert int.from_bytes(got[:32], "big") == cur[0]


def test_eval_verifier_rejections_agree_with_oracle():
    log_n, log_r, seed = 7, 3, 91
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    opp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    r = point(17, log_n)
    proof = F.vc_eval_prove(pp, cm, r)
    assert F.vc_eval_verify(pp, C, r, proof)
    blen = 1344 * log_r + 480
    y = int.from_bytes(proof[:32], "big")
    cases = {"y": ((y + 1) % I.R_INT).to_bytes(32, "big") + proof[32:]}
    for name, off in (("C_F", 100), ("L_1.T", 128 + 40), ("R_1.1", 128 + 576 + 96 + 576 + 90),
                      ("W", 128 + blen - 3), ("pi", 128 + blen + 95), ("pi_0", len(proof) - 1)):
        t = bytearray(proof)
        t[off] ^= 1
        cases[name] = bytes(t)
    for name, q in cases.items():
        assert not F.vc_eval_verify(pp, C, r, q), name
        assert not O.eval_verify(opp, C, r, q), name
    r2 = list(r)
    r2[log_n - 1] = (r2[log_n - 1] + 1) % I.R_INT
    assert not F.vc_eval_verify(pp, C, r2, proof)
    other_C = F.Commitment(pp, I.vector(5, log_n)).get()[0]
    assert not F.vc_eval_verify(pp, other_C, r, proof)
    assert not F.vc_eval_verify(pp, C, r, proof[:-1])
    big = list(r)
    big[0] = I.R_INT
    assert not F.vc_eval_verify(pp, C, big, proof)
