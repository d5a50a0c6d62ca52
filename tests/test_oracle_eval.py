"""Pins of the oracle's evaluation proof at a point (Sec. 4.4, "Compatibility with a family of
zkSNARKs"): y against the multilinear extension of the whole vector evaluated directly (and, at a
Boolean point, against the element itself), C_F and every PST proof element against their trapdoor
closed forms computed here from the definitions, and the verifier's acceptance and rejections."""
import functools
import random

import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyref as ref


def g1(k):
    return O.g1_mul(O.g1_gen(), k % ref.R)


@functools.lru_cache(maxsize=None)
def setup(log_n, log_r, seed=5):
    pp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 300, log_n)
    C, rows = O.commit(pp, m.tobytes())
    return pp, m, I.to_ints(m), C, rows


def point(seed, n):
    rnd = random.Random(seed)
    return [rnd.randrange(ref.R) for _ in range(n)]


def eq_row(j, rL):
    acc = 1
    for s, rv in enumerate(rL):
        acc = acc * (rv if (j >> s) & 1 else 1 - rv) % ref.R
    return acc


@pytest.mark.parametrize("log_n,log_r", [(4, 2), (5, 2), (5, 3), (6, 1), (6, 5)])
def test_eval_proof_closed_forms(log_n, log_r):
    pp, m, vals, C, rows = setup(log_n, log_r)
    beta, tau = pp.trapdoor()
    M, R, lc = pp.M, pp.R, pp.log_c
    r = point(log_n * 7 + log_r, log_n)
    proof = O.eval_prove(pp, m.tobytes(), C, rows, r)
    assert len(proof) == 32 + 96 + pp.bopen_len() + 96 * lc
    # y = f_m(r): the multilinear extension of all N values, evaluated from its definition
    assert int.from_bytes(proof[:32], "big") == ref.mle_eval(vals, r)
    # C_F = g1^{F(tau)}, F = sum_j T_j(r_L) f_j
    T = [eq_row(j, r[lc:]) for j in range(R)]
    Ftab = [sum(T[j] * vals[j * M + a] for j in range(R)) % ref.R for a in range(M)]
    assert proof[32:128] == g1(ref.mle_eval(Ftab, tau))
    # pi_t = g1^{q_t(tau)} with q_t the difference of the halves of F fixed to r above t
    pst = proof[128 + pp.bopen_len():]
    cur = Ftab[:]
    for idx, t in enumerate(range(lc - 1, -1, -1)):
        w = 1 << t
        q = [(cur[w + c] - cur[c]) % ref.R for c in range(w)]
        assert pst[96 * idx:96 * idx + 96] == g1(ref.mle_eval(q, tau[:t]) if t else q[0]), t
        cur = [(cur[c] + r[t] * q[c]) % ref.R for c in range(w)]
    assert cur[0] == ref.mle_eval(vals, r)
    assert O.eval_verify(pp, C, r, proof)


def test_eval_at_a_boolean_point_is_the_element():
    pp, m, vals, C, rows = setup(5, 2)
    for i in (0, 13, 31):
        r = [(i >> k) & 1 for k in range(pp.log_n)]
        proof = O.eval_prove(pp, m.tobytes(), C, rows, r)
        assert int.from_bytes(proof[:32], "big") == vals[i]
        assert O.eval_verify(pp, C, r, proof)


def test_eval_verifier_rejects():
    pp, m, vals, C, rows = setup(5, 3)
    r = point(99, pp.log_n)
    proof = O.eval_prove(pp, m.tobytes(), C, rows, r)
    assert O.eval_verify(pp, C, r, proof)
    y = int.from_bytes(proof[:32], "big")
    wrong_y = ((y + 1) % ref.R).to_bytes(32, "big") + proof[32:]
    assert not O.eval_verify(pp, C, r, wrong_y)
    r2 = list(r)
    r2[0] = (r2[0] + 1) % ref.R
    assert not O.eval_verify(pp, C, r2, proof)                      # another point
    r3 = list(r)
    r3[-1] = (r3[-1] + 1) % ref.R                                    # another row weight
    assert not O.eval_verify(pp, C, r3, proof)
    for off in (40, 128 + 30, 128 + 600, 128 + pp.bopen_len() - 5, len(proof) - 1):
        t = bytearray(proof)
        t[off] ^= 1
        assert not O.eval_verify(pp, C, r, bytes(t)), off
    other_C = O.commit(pp, I.vector(123, pp.log_n).tobytes())[0]
    assert not O.eval_verify(pp, other_C, r, proof)
    assert not O.eval_verify(pp, C, r, proof[:-1])
