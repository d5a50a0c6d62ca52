"""The serving loop: requests of mixed sizes admitted while others run (continuous batching) must
give, byte for byte, what each request gives alone with plain synchronous calls; a bad request
fails alone."""
import numpy as np
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import serve as S  # noqa: E402


def test_served_results_equal_solo_runs():
    trace = I.poisson_trace(21, 24, 2000.0, 4, 10, (1, 16, 256))
    srv = S.Server(log_n_max=10, seed=3, slots=8)
    try:
        futs = [srv.submit(I.vector(r["seed"], r["log_n"]), r["b"]) for r in trace]
        res = [f.result(timeout=240) for f in futs]
    finally:
        srv.close()
    # continuous batching: some requests were on the GPU at the same time
    assert any(a.t_admit < b.t_done and b.t_admit < a.t_done for i, a in enumerate(res) for b in res[i + 1:])
    for r, q in zip(trace, res):
        pp = srv.view(r["log_n"])
        C, rows, state = S.solo(pp, I.vector(r["seed"], r["log_n"]), r["b"])
        assert (q.C, q.rows, q.state) == (C, rows, state)
        assert q.latency > 0 and q.t_admit >= q.t_arrival
    r0 = trace[0]
    assert (res[0].C, res[0].rows) == O.commit(O.PP(r0["log_n"], 3), I.vector(r0["seed"], r0["log_n"]).tobytes())


def test_bad_request_fails_alone():
    srv = S.Server(log_n_max=6, seed=5, slots=4)
    try:
        good = I.vector(1, 6)
        bad = good.copy()
        bad[10] = np.array(I.R_LIMBS, np.uint64)
        f1, f2, f3 = srv.submit(good, 2), srv.submit(bad, 2), srv.submit(good, 8)
        assert f1.result(timeout=120).state == S.solo(srv.view(6), good, 2)[2]
        with pytest.raises(Exception):
            f2.result(timeout=120)
        assert f3.result(timeout=120).state == S.solo(srv.view(6), good, 8)[2]
        with pytest.raises(ValueError):
            srv.submit(good[:48], 1)                   # not a power of two
    finally:
        srv.close()
