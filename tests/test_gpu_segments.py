"""OpenAll for sub-arrays (Sec. 4.4) on the GPU against the oracle: setups with any split into R
segments of M elements, commitments on them, segment proofs (Step 1 only, all blocks or a block
range) byte for byte, the GPU segment verifier against the oracle's on honest and tampered inputs,
and the full OpenAll on splits other than the default (every element proof) with vc_verify_all."""
import numpy as np
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402

SPLITS = [(1, 5), (5, 1), (4, 2), (2, 6)]          # (log_r, log_c): R > M, R < M, ragged blocks


@pytest.mark.parametrize("log_r,log_c", SPLITS)
def test_split_setup_and_commit_equal_oracle(log_r, log_c):
    log_n, seed = log_r + log_c, 21
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    assert (pp.R, pp.M) == (1 << log_r, 1 << log_c)
    opp = O.PP(log_n, seed, log_r=log_r)
    assert pp.export() == opp.to_bytes()
    m = I.vector(seed + 1, log_n)
    assert F.Commitment(pp, m).get() == O.commit(opp, m.tobytes())


def test_split_views_equal_fresh_setups():
    parent = F.PP(12, 1, 23)
    for log_r, log_c in ((1, 6), (6, 1), (3, 3), (6, 6)):
        v = parent.view(log_r + log_c, log_r=log_r)
        assert v.export() == O.PP(log_r + log_c, 23, log_r=log_r).to_bytes()
    with pytest.raises(F.FlexProofsError):
        parent.view(8, log_r=7)                    # more rows than the parent has


@pytest.mark.parametrize("log_r,log_c,b", [(4, 2, 3), (5, 1, 1), (1, 5, 2), (3, 4, 8)])
def test_segment_proofs_equal_oracle_and_verify(log_r, log_c, b, schedule):
    log_n, seed = log_r + log_c, 31
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    opp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    seg = F.vc_open_segments(pp, cm, b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    M = pp.M
    for j in range(pp.R):
        p = seg.segment_proof(j)
        assert p == O.segment_proof(opp, rows, pr, j), j
        mj = m[j * M:(j + 1) * M]
        assert F.vc_verify_segment(pp, C, b, j, mj, p)
        assert O.verify_segment(opp, C, b, j, mj.tobytes(), p)
    with pytest.raises(F.FlexProofsError):
        seg.proof(0)                              # no element proofs without Step 2


def test_segment_block_range_and_rejections(schedule):
    log_r, log_c, b, seed = 4, 3, 2, 41
    log_n = log_r + log_c
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    opp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    full = F.vc_open_segments(pp, cm, b)
    part = F.vc_open_segments(pp, cm, b, 3, 2)    # blocks 3 and 4: segments 6 .. 9
    for j in range(6, 10):
        assert part.segment_proof(j) == full.segment_proof(j)
    for j in (5, 10):
        with pytest.raises(F.FlexProofsError):
            part.segment_proof(j)
    allp = F.Proofs(pp, cm, b)                    # a full OpenAll holds the same segment proofs
    assert allp.segment_proof(7) == full.segment_proof(7)
    j, M = 7, pp.M
    p = full.segment_proof(j)
    mj = m[j * M:(j + 1) * M].copy()
    assert F.vc_verify_segment(pp, C, b, j, mj, p)
    bad = mj.copy()
    bad[2, 1] ^= 8
    assert not F.vc_verify_segment(pp, C, b, j, bad, p)
    big = mj.copy()
    big[0] = np.array(I.R_LIMBS, np.uint64)
    assert not F.vc_verify_segment(pp, C, b, j, big, p)
    assert not F.vc_verify_segment(pp, C, b, j - 1, mj, p)
    assert not F.vc_verify_segment(pp, C, b, j, mj, p[:-1])
    for off in (40, 96 * 2 + 10, 96 * 2 + 576 + 95, len(p) - 2):
        t = bytearray(p)
        t[off] ^= 1
        assert not F.vc_verify_segment(pp, C, b, j, mj, bytes(t)), off
        assert not O.verify_segment(opp, C, b, j, mj.tobytes(), bytes(t)), off


@pytest.mark.parametrize("log_r,log_c,b", [(5, 2, 3), (1, 6, 1), (4, 1, 16)])
def test_full_openall_on_other_splits(log_r, log_c, b, schedule):
    """Every element proof on splits with R > M or R = 2 equals the oracle's; all verify."""
    log_n, seed = log_r + log_c, 51
    pp = F.PP(log_n, 1, seed, log_r=log_r)
    opp = O.PP(log_n, seed, log_r=log_r)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    pf = F.Proofs(pp, cm, b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r)
    assert pf.export(0, pp.N) == b"".join(pr.proof(i) for i in range(pp.N))
    ok, n = F.vc_verify_all(pf, C, m)
    assert n == pp.N and ok.all()


def test_fc_opening_at_4096_rows():
    """R = 4096 (FC length of the microbenchmark's largest n): the quotient of the fast-verification
    proof runs in chunks longer than the default; both verifiers accept the first and last segments."""
    log_r, log_c, b, seed = 12, 1, 1, 61
    pp = F.PP(log_r + log_c, 1, seed, log_r=log_r)
    opp = O.PP(log_r + log_c, seed, log_r=log_r)
    m = I.vector(seed + 1, log_r + log_c)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    for j in (0, pp.R - 1):
        p = F.vc_open_segments(pp, cm, b, j // b, 1).segment_proof(j)
        mj = m[2 * j:2 * j + 2]
        assert F.vc_verify_segment(pp, C, b, j, mj, p)
        assert O.verify_segment(opp, C, b, j, mj.tobytes(), p)
