"""Pins of the oracle's protocol layer (PST, FC, VC) against the trapdoor closed forms, the FC
round invariant, brute force (ProveOne), verification, tamper rejection and the paper's
proof-size formula."""
import functools
import os
import random

import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyref as ref


@functools.lru_cache(maxsize=None)
def setup(log_n, seed=3, dist="uniform"):
    pp = O.PP(log_n, seed)
    m = I.vector(seed + 100, log_n, dist)
    ml = m.tobytes()
    C, rows = O.commit(pp, ml)
    return pp, I.to_ints(m), ml, C, rows


@functools.lru_cache(maxsize=None)
def prover(log_n, b, seed=3):
    pp, m, ml, C, rows = setup(log_n, seed)
    pr = O.Prover(pp, ml, C, rows, b)
    pr.blocks()
    pr.step2()
    return pr


def g1(k):
    return O.g1_mul(O.g1_gen(), k % ref.R)


@pytest.mark.parametrize("log_n", [4, 5])
def test_setup_closed_forms(log_n):
    pp, *_ = setup(log_n)
    beta, tau = pp.trapdoor()
    raw = pp.to_bytes()
    M, R, lc = pp.M, pp.R, pp.log_c
    off = 0
    for t in range(lc + 1):
        for c in range(1 << t):
            assert raw[off:off + 96] == g1(ref.eq_weight(t, c, tau))
            off += 96
    assert raw[off:off + 96] == g1(beta)
    off += 96
    g2 = O.g2_gen()
    for i in range(2 * R - 1):
        assert raw[off:off + 192] == O.g2_mul(g2, pow(beta, i, ref.R))
        off += 192
    for t in range(lc):
        assert raw[off:off + 192] == O.g2_mul(g2, tau[t])
        off += 192
    assert off == len(raw)


@pytest.mark.parametrize("log_n", [4, 5])
def test_commit_closed_forms(log_n):
    pp, m, ml, C, rows = setup(log_n)
    beta, tau = pp.trapdoor()
    M = pp.M
    fj = [ref.mle_eval(m[j * M:(j + 1) * M], tau) for j in range(pp.R)]
    for j in range(pp.R):
        assert rows[96 * j:96 * j + 96] == g1(fj[j])           # C_j = g1^{f_j(tau)}
    s = sum(fj[j] * pow(beta, 2 * j, ref.R) for j in range(pp.R)) % ref.R
    e = O.pairing(O.g1_gen(), O.g2_gen())
    assert C == O.fq12_pow(e, s)                                 # C = e(g1, g2)^{sum f_j(tau) beta^{2j}}


@pytest.mark.parametrize("b,k", [(1, 0), (1, 3), (3, 1), (4, 0)])
def test_fc_round_invariant(b, k):
    pp, m, ml, C, rows = setup(4)
    _, ok = O.bopen(pp, C, rows, b, k, check_invariant=True)
    assert ok


def test_step2_closed_forms():
    log_n = 4
    pp, m, ml, C, rows = setup(log_n)
    beta, tau = pp.trapdoor()
    pr = prover(log_n, 1)
    root, rjb, gsb, dsb = pr.step2_parts()
    R, M = pp.R, pp.M
    rj = [int.from_bytes(rjb[32 * j:32 * j + 32], "big") for j in range(R)]
    assert rj == [ref.hfr("FP-rho", root + j.to_bytes(4, "big")) for j in range(R)]
    gs = [sum(rj[j] * m[j * M + a] for j in range(R)) % ref.R for a in range(M)]
    assert gsb == b"".join(v.to_bytes(32, "big") for v in gs)   # g* = sum r_j f_j
    assert dsb == g1(ref.mle_eval(gs, tau))                      # D* commits to g*
    # every PST proof element pi_t = g1^{Q_t(tau)}, Q_t = hi - lo restricted by a's top bits
    for a in range(M):
        pf = pr.proof(a)
        pst = pf[-96 * pp.log_c:]
        for idx, t in enumerate(range(pp.log_c - 1, -1, -1)):
            p = a >> (t + 1)
            w = 1 << t
            Q = [(gs[(2 * p + 1) * w + c] - gs[2 * p * w + c]) % ref.R for c in range(w)]
            assert pst[96 * idx:96 * idx + 96] == g1(ref.mle_eval(Q, tau) if t else Q[0])


@pytest.mark.parametrize("log_n,b", [(4, 1), (4, 3), (4, 4), (5, 1), (5, 4)])
def test_every_proof_verifies_and_prove_one_matches(log_n, b):
    pp, m, ml, C, rows = setup(log_n)
    pr = prover(log_n, b)
    proofs = [pr.proof(i) for i in range(pp.N)]
    assert all(O.verify_many(pp, C, b, [(i, m[i], proofs[i]) for i in range(pp.N)]))
    for i in sorted({0, pp.N - 1, 5 % pp.N, (7 * pp.M + 1) % pp.N}):
        assert O.prove_one(pp, ml, C, rows, b, i) == proofs[i]


def test_step2_independent_of_b():
    pp, *_ = setup(4)
    parts = [prover(4, b).step2_parts() for b in (1, 3, 4)]
    assert parts[0] == parts[1] == parts[2]
    # the Step-2 tail of every proof is byte-identical across b
    tail = 32 * pp.log_n + 128 * pp.log_r + 96 * pp.log_c
    for i in range(pp.N):
        ts = {prover(4, b).proof(i)[-tail:] for b in (1, 3, 4)}
        assert len(ts) == 1


def test_tampering_is_rejected():
    pp, m, ml, C, rows = setup(4)
    b = 3
    pr = prover(4, b)
    i = 6
    pf = pr.proof(i)
    assert O.verify(pp, C, b, i, m[i], pf, memo=False)
    assert not O.verify(pp, C, b, i, (m[i] + 1) % ref.R, pf, memo=False)        # flip m_i
    bad = bytearray(pf)                                                         # swap two C_a
    bad[0:96], bad[96:192] = pf[96:192], pf[0:96]
    assert not O.verify(pp, C, b, i, m[i], bytes(bad), memo=False)
    nk = 3
    Lj = 96 * nk + 576                                                          # alter L_1.1
    bad = bytearray(pf); bad[Lj:Lj + 96] = O.g1_gen()
    assert not O.verify(pp, C, b, i, m[i], bytes(bad), memo=False)
    bad = bytearray(pf); bad[-1] ^= 1                                           # PST proof byte
    assert not O.verify(pp, C, b, i, m[i], bytes(bad), memo=False)
    assert not O.verify(pp, C, b, i ^ 1, m[i], pf, memo=False)                  # wrong index


def test_zero_vector_and_identity_rows():
    # c.10.10: zero scalars give the identity; e(O, .) = 1; zero rows are allowed
    log_n = 4
    pp = O.PP(log_n, 5)
    import numpy as np
    m = np.zeros((pp.N, 4), dtype=np.uint64)
    m[3, 0] = 7
    ml = m.tobytes()
    C, rows = O.commit(pp, ml)
    assert rows[96:] == bytes(96 * (pp.R - 1))
    pr = O.Prover(pp, ml, C, rows, 2)
    pr.blocks(); pr.step2()
    vals = I.to_ints(m)
    assert all(O.verify(pp, C, 2, i, vals[i], pr.proof(i)) for i in range(pp.N))


def test_out_of_range_scalar_rejected():
    pp = O.PP(4, 5)
    import numpy as np
    m = np.zeros((pp.N, 4), dtype=np.uint64)
    m[2] = np.array(I.R_LIMBS, dtype=np.uint64)          # == r
    with pytest.raises(ValueError):
        O.commit(pp, m.tobytes())


def paper_proof_sizes():
    """The proof sizes printed in Tables tb:fc and tb:vc (tests/golden/paper_proof_sizes.txt)."""
    fc, vc = [], []
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_proof_sizes.txt")) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "fc":
                fc.append((int(w[1]), float(w[2])))
            else:
                vc.append((int(w[1]), int(w[2]), float(w[3])))
    return fc, vc


def test_proof_size_formula_reproduces_paper_tables():
    # BN_SNARK1 sizes: G1 32, G2 64, GT 384, Fr 32, digest 32 (Sec. 5, Tables tb:fc and tb:vc)
    bn = dict(g1=32, g2=64, gt=384, fr=32)
    kib = lambda v: round(v / 1024, 2)
    fc, vc = paper_proof_sizes()
    assert len(fc) == 5 and len(vc) == 10
    for log_n, b, exp in vc:
        assert kib(ref.proof_size(b, log_n, **bn)) == exp, (log_n, b)
    # FC proof alone (Table tb:fc): 2 log n GT + (2 log n + 1) G1 + 2 G2
    for n, exp in fc:
        assert kib(2 * n * 384 + (2 * n + 1) * 32 + 2 * 64) == exp, n
    # and the oracle's byte layout is that formula with BLS12-381 sizes (tower: l = l_R = l_c)
    for log_n, b in [(4, 1), (4, 4), (6, 8)]:
        pp = O.PP(log_n, 1) if log_n != 4 else setup(4)[0]
        assert pp.proof_len(b, 0) == ref.proof_size(b, log_n, g1=96, g2=192, gt=576, fr=32)


@pytest.mark.parametrize("log_n,b,k", [(4, 1, 2), (5, 3, 1), (6, 8, 0)])
def test_operation_counts_match_fc_efficiency(log_n, b, k):
    """Sec. 3's efficiency statements with n = R (the FC length).  FC.Commit takes n pairings (R
    Miller loops, one final exponentiation for their product) after the N G1 exponentiations of the
    row commitments.  FC.BOpen takes 2n pairings for the GT parts of L_j, R_j (2(R - 1) Miller loops,
    two final exponentiations per round), 2n G1 exponentiations for their G1 parts, n in G1 and n in
    G2 for the rescaling (R - 1 each) and 2n in G2 for the proof of v_l (2R - 2 terms)."""
    pp = O.PP(log_n, 3)
    m = I.vector(103, log_n).tobytes()
    R, M, lr = pp.R, pp.M, pp.R.bit_length() - 1
    O.ops_reset()
    C, rows = O.commit(pp, m)
    assert O.ops() == {"miller": R, "final_exp": 1, "g1_mul": R * M, "g2_mul": 0}
    O.ops_reset()
    O.bopen(pp, C, rows, b, k)
    assert O.ops() == {"miller": 2 * (R - 1), "final_exp": 2 * lr, "g1_mul": 3 * (R - 1), "g2_mul": 3 * (R - 1)}
