"""Pins of the oracle's OpenAll for sub-arrays (Sec. 4.4): setups with any split of N = R M into
R segments of M elements, the segment proofs (Step 1 only) and the segment verifier.

The split setup is pinned to the trapdoor closed forms (Lambda_t[c] = g1^{eq_t(c, tau)},
g2^{beta^i}, g2^{tau_t}); commitments to C_j = g1^{f_j(tau)}; a segment proof is the prefix of
every element proof of that segment (the block part and pi_{C_k}), so it is pinned to the full
verifier; the segment verifier accepts honest proofs and rejects wrong segments, wrong indices,
non-canonical values and tampered bytes."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyref as ref


def g1(k):
    return O.g1_mul(O.g1_gen(), k % ref.R)


@functools.lru_cache(maxsize=None)
def split(log_r, log_c, seed=7, b=2):
    log_n = log_r + log_c
    pp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 200, log_n)
    C, rows = O.commit(pp, m.tobytes())
    pr = O.Prover(pp, m.tobytes(), C, rows, b)
    pr.blocks()
    return pp, m, C, rows, pr


@pytest.mark.parametrize("log_r,log_c", [(1, 4), (4, 1), (3, 2), (2, 5)])
def test_split_setup_closed_forms(log_r, log_c):
    pp = O.PP(log_r + log_c, 7, log_r=log_r)
    assert (pp.R, pp.M, pp.log_r, pp.log_c) == (1 << log_r, 1 << log_c, log_r, log_c)
    beta, tau = pp.trapdoor()
    raw = pp.to_bytes()
    off = 0
    for t in range(log_c + 1):
        for c in range(1 << t):
            assert raw[off:off + 96] == g1(ref.eq_weight(t, c, tau))
            off += 96
    assert raw[off:off + 96] == g1(beta)
    off += 96
    g2 = O.g2_gen()
    for i in range(2 * pp.R - 1):
        assert raw[off:off + 192] == O.g2_mul(g2, pow(beta, i, ref.R))
        off += 192
    for t in range(log_c):
        assert raw[off:off + 192] == O.g2_mul(g2, tau[t])
        off += 192
    assert off == len(raw)


def test_split_trapdoor_is_a_prefix_of_the_default_setup():
    """The trapdoor stream draws beta, then tau_0, tau_1, ...: any split shares them."""
    beta, tau = O.PP(10, 7).trapdoor()
    for log_r, log_c in ((1, 3), (4, 5), (5, 2)):
        b2, t2 = O.PP(log_r + log_c, 7, log_r=log_r).trapdoor()
        assert b2 == beta and t2 == tau[:log_c]


@pytest.mark.parametrize("log_r,log_c", [(1, 4), (4, 1), (3, 2)])
def test_split_commit_closed_forms(log_r, log_c):
    pp, m, C, rows, _ = split(log_r, log_c)
    beta, tau = pp.trapdoor()
    vals = I.to_ints(m)
    M = pp.M
    fj = [ref.mle_eval(vals[j * M:(j + 1) * M], tau) for j in range(pp.R)]
    for j in range(pp.R):
        assert rows[96 * j:96 * j + 96] == g1(fj[j])
    s = sum(fj[j] * pow(beta, 2 * j, ref.R) for j in range(pp.R)) % ref.R
    assert C == O.fq12_pow(O.pairing(O.g1_gen(), O.g2_gen()), s)


@pytest.mark.parametrize("log_r,log_c,b", [(3, 2, 2), (4, 1, 3), (1, 4, 1)])
def test_segment_proofs_are_element_proof_prefixes_and_verify(log_r, log_c, b):
    pp, m, C, rows, _ = split(log_r, log_c, b=b)
    pr = O.Prover(pp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    vals = I.to_ints(m)
    for j in range(pp.R):
        seg = O.segment_proof(pp, rows, pr, j)
        assert len(seg) == pp.segment_proof_len(b, j // b)
        for a in (0, pp.M - 1):
            i = j * pp.M + a
            full = pr.proof(i)
            assert full[:len(seg)] == seg                     # the block part and pi_{C_k}
            assert O.verify(pp, C, b, i, vals[i], full, memo=False)
        assert O.verify_segment(pp, C, b, j, m[j * pp.M:(j + 1) * pp.M].tobytes(), seg)


def test_segment_verifier_rejects():
    pp, m, C, rows, pr = split(3, 2, b=2)
    b, j = 2, 5
    seg = O.segment_proof(pp, rows, pr, j)
    mj = m[j * pp.M:(j + 1) * pp.M].copy()
    assert O.verify_segment(pp, C, b, j, mj.tobytes(), seg)
    wrong = mj.copy()
    wrong[1, 0] ^= 1
    assert not O.verify_segment(pp, C, b, j, wrong.tobytes(), seg)         # another segment value
    big = mj.copy()
    big[0] = np.array(I.R_LIMBS, np.uint64)
    assert not O.verify_segment(pp, C, b, j, big.tobytes(), seg)           # value r: not canonical
    assert not O.verify_segment(pp, C, b, j - 1, mj.tobytes(), seg)        # another index, same block
    assert not O.verify_segment(pp, C, b, j, mj.tobytes(), seg[:-1])       # wrong length
    for off in (95, 96 * 2 + 100, 96 * 2 + 576 + 50, len(seg) - 1):       # C_a, L_1.T, L_1.1, W
        t = bytearray(seg)
        t[off] ^= 1
        assert not O.verify_segment(pp, C, b, j, mj.tobytes(), bytes(t)), off
    other_C = O.commit(pp, I.vector(77, pp.log_n).tobytes())[0]
    assert not O.verify_segment(pp, other_C, b, j, mj.tobytes(), seg)
