"""Host-side logic of the serving loop (no GPU): admission order, slots, the memory budget,
overlap of running jobs, failure isolation and shutdown, with a fake backend whose jobs finish
after a set time."""
import threading
import time

import numpy as np
import pytest

from paper_2601_03031_gb300 import serve as S


class FakeBackend:
    def __init__(self, dur=0.02, fail_b=None):
        self.dur, self.fail_b = dur, fail_b
        self.started, self.lock = [], threading.Lock()

    def free_memory(self):
        return 1 << 40

    def view(self, log_n):
        return log_n

    def start(self, req, slot):
        if req.b == self.fail_b and req.log_n == 5:
            raise RuntimeError("enqueue failed")
        with self.lock:
            self.started.append((time.perf_counter(), req.log_n, req.b, slot))
        return {"t": time.perf_counter() + self.dur * req.log_n / 4, "req": req}

    @staticmethod
    def ready(job):
        return time.perf_counter() >= job["t"]

    def finish(self, job):
        req = job["req"]
        if req.b == self.fail_b:
            raise RuntimeError("job failed")
        return b"C%d" % req.log_n, b"rows", bytes(req.m[:2].tobytes())


def vec(log_n, fill=1):
    return np.full((1 << log_n, 4), fill, np.uint64)


def test_results_slots_and_overlap():
    be = FakeBackend()
    srv = S.Server(log_n_max=10, slots=3, hbm_budget=1 << 40, backend=be)
    futs = [srv.submit(vec(4 + i % 5, i), 1 + i % 2) for i in range(12)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    for i, r in enumerate(res):
        assert r.state == vec(4 + i % 5, i)[:2].tobytes() and r.log_n == 4 + i % 5
        assert r.t_arrival <= r.t_admit <= r.t_done
    assert srv.peak_running == 3                        # slots bound the running jobs ...
    assert any(a.t_admit < b.t_done and b.t_admit < a.t_done for i, a in enumerate(res) for b in res[i + 1:])
    assert [s[1] for s in be.started] == [4 + i % 5 for i in range(12)]   # ... and admission is FIFO


def test_memory_budget_serialises_big_jobs():
    need = S.footprint_bytes(10, 1)
    be = FakeBackend()
    srv = S.Server(log_n_max=10, slots=8, hbm_budget=int(1.5 * need), backend=be)
    futs = [srv.submit(vec(10), 1) for _ in range(3)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    assert srv.peak_running == 1                        # two of them never fit together
    order = sorted(res, key=lambda r: r.t_admit)
    assert all(order[i].t_done <= order[i + 1].t_admit for i in range(2))


def test_failures_stay_with_their_request():
    be = FakeBackend(fail_b=2)
    srv = S.Server(log_n_max=8, slots=2, hbm_budget=1 << 40, backend=be)
    ok1, bad_start, bad_run, ok2 = (srv.submit(vec(4), 1), srv.submit(vec(5), 2), srv.submit(vec(6), 2),
                                    srv.submit(vec(4), 1))
    assert ok1.result(timeout=30).log_n == 4 and ok2.result(timeout=30).log_n == 4
    with pytest.raises(RuntimeError, match="enqueue failed"):
        bad_start.result(timeout=30)
    with pytest.raises(RuntimeError, match="job failed"):
        bad_run.result(timeout=30)
    with pytest.raises(ValueError):
        srv.submit(vec(4)[:10], 1)
    with pytest.raises(ValueError):
        srv.submit(vec(4), 5)                           # b > R = 4
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit(vec(4), 1)


def test_worker_crash_fails_pending_futures():
    class Broken(FakeBackend):
        @staticmethod
        def ready(job):
            raise KeyError("poll broke")
    srv = S.Server(log_n_max=8, slots=1, hbm_budget=1 << 40, backend=Broken())
    futs = [srv.submit(vec(4), 1) for _ in range(3)]
    for f in futs:
        with pytest.raises(RuntimeError, match="worker stopped"):
            f.result(timeout=30)
