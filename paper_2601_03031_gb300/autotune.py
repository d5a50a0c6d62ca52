"""Schedule autotuner: chooses the engine-choice limits (fp_set_engine_limits) and the MSM window for a
workload by timing it on the GPU, and keeps the choices in a JSON table so that later processes
reuse them without tuning again.

A workload is a callable that enqueues one run and returns something to keep alive until the run
completes (the tuner synchronises the device around each timed run).  Tuning is coordinate descent
over groups of limits: each group has a few settings (from "latency engines for few items" to
"one thread per item"), every setting of a group is timed with the other groups fixed at their
current best, and the pass repeats until no group changes.  Every limit setting gives the same
bytes, so tuning never changes a result, only the time.

Keys name the workload shape, e.g. ``proveall:log_n=16,b=256`` or ``batch:<mix>`` for a job mix
(``batch_key``); the table maps each key to its limits, its time and the trials that chose them.
"""
from __future__ import annotations

import json
import os
import time

from . import _lib as F

UNLIMITED = 0xFFFFFFFF

# settings of each group of limits: latency engines up to the default sizes, fewer latency engines,
# and one thread per item (0: no launch is small enough for a block or a warp)
GROUPS = {
    "miller": [{}, {"miller_block_max": 256, "miller_warp_max": 4096}, {"miller_block_max": 0, "miller_warp_max": 0},
               {"miller_block_max": 0}],
    "final_exp": [{}, {"fe_block_max": 0}, {"fe_block_max": 0, "fe_warp_max": 64}, {"fe_block_max": 0, "fe_warp_max": 0}],
    "folds": [{}, {"fold_warp_max": 1024, "wterm_warp_max": 1024}, {"fold_warp_max": 0, "wterm_warp_max": 0}],
    "commit": [{}, {"commit_block_max": 0}, {"commit_block_max": 0, "commit_warp_max": 0}],
    "pairs": [{}, {"pair_block_max": 256}, {"pair_block_max": 0}],
}
MSM_CHUNKS = [1 << 15, 1 << 16, 1 << 17, 1 << 18]
MSM_SEGMENTS = [1 << 13, 1 << 15, 1 << 17]


def default_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "flexproofs", "tuning.json")


def proveall_key(log_n: int, b: int) -> str:
    return f"proveall:log_n={log_n},b={b}"


def batch_key(shapes) -> str:
    """Key of a job mix: the multiset of (log N, b) of its jobs."""
    from collections import Counter
    c = Counter((int(ln), int(b)) for ln, b in shapes)
    return "batch:" + ";".join(f"{ln}/{b}x{n}" for (ln, b), n in sorted(c.items()))


def load_table(path: str | None = None) -> dict:
    path = path or default_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_entry(key: str, entry: dict, path: str | None = None) -> None:
    path = path or default_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    table = load_table(path)
    table[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(key: str, path: str | None = None) -> bool:
    """Set the stored limits of `key` if the table has them; returns whether it did."""
    entry = load_table(path).get(key)
    if not entry:
        return False
    F.set_engine_limits(entry["limits"])
    return True


def time_workload(fn, reps: int = 3) -> float:
    """Best host wall time (s) of fn() over `reps` runs, device synchronised around each."""
    import torch
    keep = fn()                      # warm-up (and first-use set-up)
    torch.cuda.synchronize()
    del keep
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        keep = fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
        del keep
    return best


def tune_engines(key: str, fn, path: str | None = None, reps: int = 3, groups=None, max_passes: int = 2) -> dict:
    """Coordinate descent over the limit groups for workload fn; stores and applies the best limits.
    Returns the table entry: {"limits", "ms", "default_ms", "trials"}."""
    groups = groups or GROUPS
    choice = {g: 0 for g in groups}

    def limits_of(ch):
        lim = {}
        for g, i in ch.items():
            lim.update(groups[g][i])
        return lim

    trials = []

    def measure(ch):
        lim = limits_of(ch)
        F.set_engine_limits(lim)
        t = time_workload(fn, reps)
        trials.append({"limits": lim, "ms": t * 1e3})
        return t

    try:
        best_t = measure(choice)
        default_ms = best_t * 1e3
        for _ in range(max_passes):
            changed = False
            for g in groups:
                for i in range(len(groups[g])):
                    if i == choice[g]:
                        continue
                    trial = dict(choice, **{g: i})
                    t = measure(trial)
                    if t < 0.98 * best_t:          # a clear win only: timing noise is ~1-2 %
                        best_t, choice, changed = t, trial, True
            if not changed:
                break
    finally:
        F.set_engine_limits(None)
    entry = {"limits": limits_of(choice), "ms": best_t * 1e3, "default_ms": default_ms, "trials": trials}
    save_entry(key, entry, path)
    F.set_engine_limits(entry["limits"])
    return entry


def tune_msm(bases, k_dev, nbatch: int = 1, stream=None, path: str | None = None, reps: int = 3) -> dict:
    """MSM schedule for (n, nbatch): the window by fp_msm_autotune, then the bucket-pass chunk count and
    the reduction's segment cap by timing; stores {"window", "msm_chunks", "msm_segment_threads", "ms"}
    under "msm:n=..,nbatch=.." and leaves the best limits set."""
    import torch
    n = k_dev.shape[0] // nbatch
    window, _ = F.msm_autotune(bases, k_dev, nbatch, stream)
    out = torch.zeros(96 * nbatch, dtype=torch.uint8, device="cuda")
    base = F.engine_limits()
    best = None
    trials = []
    for ch in MSM_CHUNKS:
        for sg in MSM_SEGMENTS:
            F.set_engine_limits(dict(base, msm_chunks=ch, msm_segment_threads=sg))
            t = time_workload(lambda: F.msm_g1(bases, k_dev, nbatch, 0, stream, out), reps)
            trials.append({"msm_chunks": ch, "msm_segment_threads": sg, "ms": t * 1e3})
            if best is None or t < best[0]:
                best = (t, ch, sg)
    entry = {"window": window, "msm_chunks": best[1], "msm_segment_threads": best[2], "ms": best[0] * 1e3,
             "limits": dict(base, msm_chunks=best[1], msm_segment_threads=best[2]), "trials": trials}
    save_entry(f"msm:n={n},nbatch={nbatch}", entry, path)
    F.set_engine_limits(entry["limits"])
    return entry
