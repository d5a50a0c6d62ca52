"""bench.py's multi-process path (N > 1 under torchrun) on the CPU with two gloo ranks.

Each rank proves its own vector (replicas: no collective on the data path); the only collective is
the max over ranks of the timed region, and the whole-job value is all ranks' proofs over that
time.  The reference arm runs on rank 0 only; the other ranks exit without output.
"""
import argparse
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total_ms = bench.slowest_rank_ms(10.0 + 5.0 * rank, world, dist, "cpu")
    q.put((rank, total_ms, bench.job_proofs_per_s(world, 1 << 16, total_ms / 5), bench.replica_seed(1, rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_value_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]                      # the slowest rank's time
    assert res[0][2] == res[1][2] == 2 * (1 << 16) / 3e-3          # 2 replicas x N per 3 ms step
    assert len({r[3] for r in res}) == 2                           # each replica its own vector


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5, 1) == 12.5
    assert bench.job_proofs_per_s(1, 1 << 16, 35.0) == (1 << 16) / 35e-3


def test_reference_arm_only_on_rank_0(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(log_n=16, b=256, seed=1, steps=1, warmup=0)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
