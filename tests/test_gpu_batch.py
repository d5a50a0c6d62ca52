"""Batched OpenAll over one resident SRS: SRS views, asynchronous commitments, and
vc_prove_all_batch (concurrent job streams, optionally one CUDA graph) against single calls and
the oracle.  Exact arithmetic: every byte must match."""
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


def b_for(log_n: int) -> int:
    """b = min(R, nearest power of two to log^2 N), the batched workload's rule."""
    return min(1 << (log_n // 2), I.nearest_pow2(log_n * log_n))


def state(pf) -> bytes:
    buf = np.zeros(pf.state_size(), np.uint8)
    pf.state_into(buf)
    return buf.tobytes()


@pytest.mark.parametrize("log_n", [2, 4, 5, 7, 10])
def test_view_equals_fresh_setup(log_n):
    parent = F.PP(10, 1, 13)
    view = parent.view(log_n)
    assert (view.R, view.M, view.N) == (1 << (log_n // 2), 1 << (log_n - log_n // 2), 1 << log_n)
    assert view.export() == O.PP(log_n, 13).to_bytes()


def test_commit_async_status():
    pp = F.PP(4, 1, 3)
    good = I.vector(5, 4)
    cm = F.Commitment(pp, good, sync=False)
    assert cm.status() == 0
    assert cm.get() == F.Commitment(pp, good).get()
    bad = good.copy()
    bad[3] = np.array(I.R_LIMBS, np.uint64)
    assert F.Commitment(pp, bad, sync=False).status() == 6


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_calls_and_oracle(use_graph, schedule):
    seed = 17
    parent = F.PP(10, 1, seed)
    sizes = [4, 5, 6, 7, 8, 10, 4, 9, 6, 5]
    views = {ln: parent.view(ln) for ln in set(sizes)}
    vecs = [I.vector(seed + 100 + j, ln) for j, ln in enumerate(sizes)]
    cms = [F.Commitment(views[ln], m, sync=False) for ln, m in zip(sizes, vecs)]
    assert all(cm.status() == 0 for cm in cms)
    jobs = [(cm, b_for(ln)) for cm, ln in zip(cms, sizes)]
    outs = F.vc_prove_all_batch(jobs, use_graph=use_graph)
    for (cm, b), pf, ln, m in zip(jobs, outs, sizes, vecs):
        single = F.Proofs(cm.pp, cm, b)
        assert state(pf) == state(single)
        assert pf.export(0, cm.pp.N) == single.export(0, cm.pp.N)
    # one job of each odd/even shape against the oracle, every proof
    for j in (1, 2):
        ln, m = sizes[j], vecs[j]
        cm, b = jobs[j]
        opp = O.PP(ln, seed)
        C, rows = O.commit(opp, m.tobytes())
        assert cm.get() == (C, rows)
        pr = O.Prover(opp, m.tobytes(), C, rows, b)
        pr.blocks()
        pr.step2()
        _state.assert_equal(state(outs[j]), pr.state(), cm.pp.R, cm.pp.M, pr.K, opp.log_r)
        assert outs[j].export(0, cm.pp.N) == b"".join(pr.proof(i) for i in range(cm.pp.N))


def test_batched_workload_64_jobs_sampled(schedule):
    """64 jobs, log N uniform in 8..18 by seed, b = min(R, nearestpow2(log^2 N)), one SRS for 2^18:
    the graph-captured batch equals single calls (shared state of every job), and the smallest
    job's proofs equal the oracle's."""
    jobs_spec = I.batched_jobs(4, 64, 8, 18)
    parent = F.PP(18, 1, 4)
    views = {}
    cms = []
    for spec in jobs_spec:
        ln = spec["log_n"]
        if ln not in views:
            views[ln] = parent.view(ln)
        cms.append(F.Commitment(views[ln], I.vector(spec["seed"], ln), sync=False))
    jobs = [(cm, spec["b"]) for cm, spec in zip(cms, jobs_spec)]
    assert [b for _, b in jobs] == [b_for(s["log_n"]) for s in jobs_spec]
    outs = F.vc_prove_all_batch(jobs, use_graph=True)
    for (cm, b), pf in zip(jobs, outs):
        assert state(pf) == state(F.Proofs(cm.pp, cm, b))
    j = min(range(64), key=lambda q: jobs_spec[q]["log_n"])
    ln, cm, b = jobs_spec[j]["log_n"], jobs[j][0], jobs[j][1]
    opp = O.PP(ln, 4)
    m = I.vector(jobs_spec[j]["seed"], ln)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks([0])
    pr.step2()
    _state.assert_equal(state(outs[j]), pr.state(), cm.pp.R, cm.pp.M, pr.K, opp.log_r, [0])
    for i in (0, 7, cm.pp.M - 1):
        assert outs[j].proof(i) == pr.proof(i)
