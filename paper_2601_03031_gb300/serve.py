"""Serving loop for OpenAll requests with continuous batching.

A Server keeps one SRS resident (vc_setup for the largest size, vc_pp_view for the smaller ones)
and a worker thread that admits requests in arrival order whenever a slot and enough device
memory are free: each admitted job gets its own CUDA stream, its commitment and OpenAll are only
enqueued there (vc_commit_async, vc_prove_all), so jobs admitted while others run overlap on the
GPU, and the worker polls completion events.  A finished job's proof state is copied into pinned
host memory and handed to the request's future; its device memory is released stream-ordered.

Everything a job computes runs in the library's kernels; this module only schedules.  More
streams than the CUDA default of 8 hardware queues help jobs overlap: set
CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32) before the process creates its CUDA context.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


def footprint_bytes(log_n: int, b: int) -> int:
    """Upper bound of the device memory one job allocates (commitment + OpenAll), from the sizes of
    its buffers: vector copies, MSM scratch, Merkle trees, fold tree, Step 1's per-block tables."""
    lr = log_n // 2
    lc = log_n - lr
    R, M = 1 << lr, 1 << lc
    N = R * M
    K = (R + b - 1) // b
    KR = K * R
    commit = N * 32 * 3 + N * 2 * 20 * 4 + R * (96 * 2 + 576 * 2) + (1 << 22)
    step2 = R * (2 * M - 1) * 32 + (2 * R - 1) * 32 + (2 * R - 1) * M * 32 + (2 * R - 1) * 192 + lc * M * 72
    step1 = KR * (96 + 192 + 32 + 576 * 3 // 2 + 144 * 3 // 2) + K * (2 * R) * (32 * 2 + 288 * 3 // 2)
    blocks = K * (lr * 1344 + 480)
    return int(commit + step2 + step1 + blocks + (8 << 20))


@dataclass
class Result:
    """What a request gets back: the commitment C (576 B), the row commitments (R x 96 B) and the
    OpenAll proof state (vc_proofs_state bytes), plus timestamps (time.perf_counter seconds)."""
    log_n: int
    b: int
    C: bytes
    rows: bytes
    state: bytes
    t_arrival: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass(eq=False)
class _Request:
    m: np.ndarray
    b: int
    log_n: int
    t_arrival: float
    future: Future = field(default_factory=Future)


@dataclass(eq=False)
class _Running:
    req: _Request
    slot: int
    need: int
    t_admit: float
    job: object


class GpuBackend:
    """Runs jobs through the library: one resident SRS, one CUDA stream per slot."""

    def __init__(self, log_n_max: int, seed: int, slots: int):
        import torch
        from . import _lib as F
        self.torch, self.F = torch, F
        self.pp = F.PP(log_n_max, 1, seed)
        self.views = {log_n_max: self.pp}
        self.streams = [torch.cuda.Stream() for _ in range(slots)]

    def free_memory(self) -> int:
        return int(self.torch.cuda.mem_get_info()[0])

    def view(self, log_n: int):
        if log_n not in self.views:
            self.views[log_n] = self.pp.view(log_n)
        return self.views[log_n]

    def start(self, req: _Request, slot: int):
        torch, F = self.torch, self.F
        st = self.streams[slot]
        pp = self.view(req.log_n)
        host = torch.from_numpy(req.m.view(np.int64)).pin_memory()
        with torch.cuda.stream(st):
            dev = host.to("cuda", non_blocking=True)
        cm = F.Commitment(pp, dev, stream=st, sync=False)
        pf = F.Proofs(pp, cm, req.b, stream=st)
        done = torch.cuda.Event()
        done.record(st)
        return {"host": host, "dev": dev, "cm": cm, "pf": pf, "done": done}

    @staticmethod
    def ready(job) -> bool:
        return job["done"].query()

    def finish(self, job):
        cm, pf = job["cm"], job["pf"]
        st = cm.status()
        if st != 0:
            raise self.F.FlexProofsError("vc_commit", st)
        C, rows = cm.get()
        buf = self.torch.empty(pf.state_size(), dtype=self.torch.uint8).pin_memory()
        pf.state_into(buf)
        job.clear()                     # handles are released stream-ordered
        return C, rows, bytes(buf.numpy())


class Server:
    """submit(m, b) -> Future[Result].  m: N x 4 little-endian uint64 canonical Fr values, N = 2^n
    with 2 <= n <= log_n_max; 1 <= b <= R = 2^floor(n/2).

    Admission is in arrival order: the head request starts as soon as a slot is free and its
    device-memory bound (footprint_bytes) fits in the budget next to the running jobs (a request
    that alone exceeds the budget starts when nothing else runs)."""

    def __init__(self, log_n_max: int = 20, seed: int = 0, slots: int = 32, hbm_budget: int | None = None,
                 poll_s: float = 2e-4, backend=None):
        self.backend = backend if backend is not None else GpuBackend(log_n_max, seed, slots)
        self.log_n_max = log_n_max
        self.budget = int(hbm_budget if hbm_budget is not None else 0.7 * self.backend.free_memory())
        self.slots = slots
        self.poll_s = poll_s
        self.free_slots = list(range(slots))
        self.pending: collections.deque[_Request] = collections.deque()
        self.running: list[_Running] = []
        self.used = 0
        self.peak_running = 0
        self.lock = threading.Condition()
        self.closed = False
        self.error: Exception | None = None
        self.worker = threading.Thread(target=self._loop, name="flexproofs-server", daemon=True)
        self.worker.start()

    def view(self, log_n: int):
        return self.backend.view(log_n)

    def submit(self, m: np.ndarray, b: int, t_arrival: float | None = None) -> Future:
        m = np.ascontiguousarray(m, dtype=np.uint64).reshape(-1, 4)
        n = m.shape[0]
        log_n = n.bit_length() - 1
        if n != 1 << log_n or not 2 <= log_n <= self.log_n_max:
            raise ValueError(f"vector length {n} is not a power of two in [4, 2^{self.log_n_max}]")
        if not 1 <= b <= 1 << (log_n // 2):
            raise ValueError(f"b = {b} outside [1, R]")
        req = _Request(m, b, log_n, time.perf_counter() if t_arrival is None else t_arrival)
        with self.lock:
            if self.closed:
                raise RuntimeError("server closed")
            self.pending.append(req)
            self.lock.notify()
        return req.future

    def close(self):
        with self.lock:
            self.closed = True
            self.lock.notify()
        self.worker.join()

    # ------------------------------------------------------------------ worker
    def _loop(self):
        try:
            self._serve()
        except Exception as e:          # never leave futures hanging: fail everything still queued
            self.error = e
            with self.lock:
                self.closed = True
                waiting = list(self.pending) + [r.req for r in self.running]
                self.pending.clear()
                self.running = []
            for req in waiting:
                if not req.future.done():
                    req.future.set_exception(RuntimeError(f"server worker stopped: {e!r}"))

    def _select(self) -> list[_Request]:
        admit, extra = [], 0
        while self.pending and len(admit) < len(self.free_slots):
            need = footprint_bytes(self.pending[0].log_n, self.pending[0].b)
            if (self.running or admit) and self.used + extra + need > self.budget:
                break                   # in arrival order: wait for memory to free up
            admit.append(self.pending.popleft())
            extra += need
        return admit

    def _serve(self):
        while True:
            with self.lock:
                while not self.pending and not self.running and not self.closed:
                    self.lock.wait()
                if self.closed and not self.pending and not self.running:
                    return
                admit = self._select()
            for req in admit:
                slot = self.free_slots.pop()
                need = footprint_bytes(req.log_n, req.b)
                t_admit = time.perf_counter()
                try:
                    job = self.backend.start(req, slot)
                except Exception as e:
                    self.free_slots.append(slot)
                    req.future.set_exception(e)
                    continue
                self.used += need
                self.running.append(_Running(req, slot, need, t_admit, job))
            self.peak_running = max(self.peak_running, len(self.running))
            finished = [r for r in self.running if self.backend.ready(r.job)]
            if finished:
                done_ids = {id(r) for r in finished}
                self.running = [r for r in self.running if id(r) not in done_ids]
            for r in finished:
                try:
                    C, rows, state = self.backend.finish(r.job)
                    r.req.future.set_result(Result(r.req.log_n, r.req.b, C, rows, state, r.req.t_arrival,
                                                   r.t_admit, time.perf_counter()))
                except Exception as e:  # the request fails, the server keeps serving
                    r.req.future.set_exception(e)
                finally:
                    r.job = None
                    self.used -= r.need
                    self.free_slots.append(r.slot)
            if not admit and not finished:
                time.sleep(self.poll_s)


def solo(pp, m: np.ndarray, b: int) -> tuple[bytes, bytes, bytes]:
    """The same request run alone with plain synchronous calls: (C, rows, proof state)."""
    from . import _lib as F
    cm = F.Commitment(pp, m)
    pf = F.Proofs(pp, cm, b)
    C, rows = cm.get()
    buf = np.zeros(pf.state_size(), np.uint8)
    pf.state_into(buf)
    return C, rows, buf.tobytes()
