"""Benchmark of the FlexProofs all-proofs pass (VC.Commit + VC.OpenAll) on GB300.

Workload (default): N = 2^16 uniform Fr values (BLS12-381 scalar field), batch size b = 256
(= log^2 N), seeded synthetic input resident in HBM.  One step = one pass of the whole hot path:
Commit (row MSMs + FC multi-pairing) followed by OpenAll (Step 1 for every block, Step 2).
Metric: proofs/s = N / (step time).  The paper reports 0.23 s for this (N, b) point, but on the
BN_SNARK1 curve with a single CPU thread, so there is no like-for-like baseline (vs_baseline null).

N > 1 (torchrun): every rank proves its own vector (replicas, weak scaling, no collective on the
data path); value = all ranks' proofs / max-over-ranks time.

--impl reference times the CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware queues than the default 8, so that concurrent job streams overlap (batched and
# served workloads); must be set before the CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

# Fq multiplications per unit operation, from the operation counts of efficient textbook formulas
# (an Fq multiplication is one 12-limb CIOS Montgomery product = 4 * 12^2 = 576 32-bit
# multiply-adds).  These are ALGORITHMIC counts: the kernels' own formulas may do more.
FQ_MUL_IMAD = 4 * 12 * 12
FQ_MULS = {
    "miller_loop": 7135,     # 62 Fq12 sqr + 63 doubling steps + 5 addition steps, with their lines
    "final_exp": 10120,      # easy part (Fq12 inverse) + h1 and three |x| cyclotomic exponentiations
    "g1_mul": 2000,          # GLV: 128 Jacobian doublings (7) + ~96 mixed additions (11)
    "g2_mul": 3300,          # GLS: 64 doublings + ~60 mixed additions over Fq2, 15-point table
    "msm_madd": 10,          # XYZZ mixed addition (8M + 2S), one per bucket entry
    # one pair of a 4-pair multi-Miller loop: the 62 Fq12 squarings (36 Fq products each) are shared
    # by the 4 pairs, so a pair costs 7135 - 3/4 x 62 x 36
    "miller_loop_multi4": 7135 - 3 * 62 * 36 // 4,
    "g2_msm_madd": 30,       # XYZZ mixed addition over Fq2 (8M + 2S), 3 Fq products per Fq2 product
    # comb folds of a point of A and of v (k_step1.cu): 64 table entries and the L half added with
    # complete additions (12 Fq products on G1, 12 Fq2 products of 3 on G2)
    "comb_fold": 65 * 12 + 65 * 36,
    # their chains: 127 G1 and 63 G2 complete doublings (6M + 2S)
    "comb_chain": 127 * 8 + 63 * 8 * 3,
    # their tables: per G1 window 10 additions and 3 products by omega, per G2 position 7 additions
    # and 7 psi maps (2 Fq2 products each)
    "comb_tab": 64 * (10 * 12 + 3) + 64 * (7 * 36 + 7 * 6),
    # a commitment term by the setup's combs (k_lamcomb.cu): 32 mixed additions (7M + 4S)
    "lamc_term": 32 * 11,
    # a W term by the setup's G2 combs: 64 position entries summed, 63 complete additions over Fq2
    "w_comb_term": 63 * 36,
}


def _cyc_exp_rounds(e: int) -> int:
    """Product rounds of a square-and-multiply exponentiation by e (squarings + multiplications)."""
    return (e.bit_length() - 1) + (bin(e).count("1") - 1)


def _wnaf4_exp_rounds(e: int) -> int:
    """Product rounds of an exponentiation by e on its width-4 NAF: base^2, 3, 5, 7, then a squaring
    per digit below the top one and a product per nonzero digit below it."""
    digits = []
    while e:
        d = 0
        if e & 1:
            d = e % 16
            d = d - 16 if d >= 8 else d
            e -= d
        digits.append(d)
        e >>= 1
    return 4 + (len(digits) - 1) + sum(1 for d in digits[:-1] if d)


X_ABS = 0xd201000000010000                   # |x| of BLS12-381 (x < 0)
H1 = (X_ABS + 1) ** 2 // 3                   # h1 = (x - 1)^2 / 3
# Sequential Fq-product rounds on one launch's critical path in the lane-parallel engines: every
# round waits for one dependent Montgomery product, so rounds x the measured product latency is a
# lower bound on the launch time (the linear combinations between rounds and the one-lane
# binary-gcd inversions are left out, so the bound is optimistic).
CRITICAL_ROUNDS = {
    # easy part 8 rounds (n, two Frobenius^2, u, n u, c^2, c^2 u, t) + 5 products of the Fq2 inverse,
    # g 2, hard part: h1 on its width-4 NAF and 3 |x| exponentiations (cyclotomic squarings split over
    # the block's warps, products one per lane) + 6 Frobenius / product rounds
    "k_final_exp_c": 8 + 5 + 2 + _wnaf4_exp_rounds(H1) + 3 * _cyc_exp_rounds(X_ABS) + 6,
    # pipelined Miller loop: a priming round, 63 doubling steps of 2 rounds, 5 addition steps of 4
    # each followed by a priming round
    "k_round_miller_c": 1 + 63 * 2 + 5 * (4 + 1),
    "k_commit_miller_c": 1 + 63 * 2 + 5 * (4 + 1),
    # G1 by 8-lane groups, 2-bit joint GLV windows: 13 table formulas + 64 x (2 doublings + 1 addition),
    # 2 phases each, then the addition of A_L and the conversion (longer than the warp G2 chain)
    "k_fold_w": (13 + 64 * 3) * 2 + 2 + 3,
    # comb folds (rounds of at most 256 points): the G2 warp's 7 additions of table entries, 3 tree
    # levels and the addition of v_L, 2 phases each, then the conversion (the G1 groups' 3 + 4 + 1
    # additions are shorter)
    "k_fold_c": (7 + 3 + 1) * 2 + 3,
    # comb chains beside the round: 127 G1 doublings of 2 phases
    "k_comb_chain": 127 * 2,
    "k_sparse_g": (13 + 64 * 3) * 2 + 2,
}
# of those rounds, the ones whose product is split over a block's four warps (fq_split.cuh): the
# cyclotomic squarings (h1's NAF has one digit more than h1 has bits: base^2 and one per lower digit)
SPLIT_ROUNDS = {"k_final_exp_c": (H1.bit_length() + 1) + 3 * (X_ABS.bit_length() - 1)}
# the kernels of Step 1's round chain (the rest of a round runs beside it)
CHAIN_KERNELS = ("k_final_exp_c", "k_round_miller_c", "k_fold_c", "k_challenge2")


FOLD_COMB_MAX = 256           # rounds with at most this many fold points use the comb folds
LAM_COMB_MAX_M = 1024         # setups with M <= this commit by the fixed-base combs of their bases
G2_COMB_MAX_R = 1024          # setups with R <= this keep the W proofs' comb tables

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# kernel at this workload, keyed by (log N, b, kernel); an entry is removed when its kernel changes
NCU_TRAFFIC = {
    (16, 256, "k_round_miller_c"): 277e3,
    (16, 256, "k_lamc_sum"): 310e6,
}


def step_units(log_n: int, b: int, msm_window: int, msm_window_g2: int = 16, lim: dict | None = None) -> dict:
    """Per kernel: (unit, units processed per step) for one Commit + OpenAll step.  `lim` is the
    library's engine-choice limits (fp_get_engine_limits: the launch sizes at which a kernel moves
    from a block to a warp to a thread per item, chosen as the library's launchers do); None reads
    the current ones."""
    if lim is None:
        from paper_2601_03031_gb300 import _lib as F
        lim = F.engine_limits()
    lr = log_n // 2
    lc = log_n - lr
    R, M = 1 << lr, 1 << lc
    K = (R + b - 1) // b
    hs = [R >> j for j in range(1, lr + 1)]
    W = -(-129 // msm_window)
    W2 = -(-65 // msm_window_g2)
    w_msm = K * R * 2 > 4096 and K >= 8         # the W proofs by one batched G2 MSM

    def engine(n, block_max, warp_max):         # "c" a block, "w" a warp, "t" a thread per item
        if n > warp_max and n > block_max:
            return "t"
        return "c" if n <= block_max else "w"

    mb, mw, mg = lim["miller_block_max"], lim["miller_warp_max"], lim["miller_group_min"]
    miller = {"c": 0, "w": 0, "t": 0, "t4": 0}
    for h in hs:
        n = K * 2 * h
        e = engine(n, mb, mw)
        miller["t4" if e == "t" and h >= 4 and n >= mg else e] += n
    fe = {"c": 0, "w": 0, "t": 0}
    fe[engine(1, lim["fe_block_max"], lim["fe_warp_max"])] += 1                  # Commit's one
    fe[engine(2 * K, lim["fe_block_max"], lim["fe_warp_max"])] += 2 * K * lr     # two per block and round
    cm = {"c": 0, "w": 0, "t": 0}
    cm[engine(R, lim["commit_block_max"], lim["commit_warp_max"])] += R
    comb = sum(K * h for h in hs if K * h <= FOLD_COMB_MAX)
    fw = lim["fold_warp_max"]
    w_terms = K * (2 * R - 2) if not w_msm and R > G2_COMB_MAX_R else 0
    return {
        "k_final_exp_c": ("final_exp", fe["c"]),
        "k_final_exp_w": ("final_exp", fe["w"]),
        "k_final_exp_t": ("final_exp", fe["t"]),
        "k_round_miller_c": ("miller_loop", miller["c"]),
        "k_round_miller_w": ("miller_loop", miller["w"]),
        "k_step1_miller_multi": ("miller_loop_multi4", miller["t4"]),
        "k_step1_miller": ("miller_loop", miller["t"]),
        "k_commit_miller_c": ("miller_loop", cm["c"]),
        "k_commit_miller_w": ("miller_loop", cm["w"]),
        "k_commit_miller": ("miller_loop", cm["t"]),
        "k_sparse_g": ("g1_mul", sum(K * min(b, 2 * h) for h in hs)),
        "k_fold_c": ("comb_fold", comb),
        "k_comb_chain": ("comb_chain", comb),
        "k_comb_tab": ("comb_tab", comb),
        "k_fold_w": (("g1_mul", "g2_mul"), sum(K * h for h in hs if FOLD_COMB_MAX < K * h <= fw)),
        "k_fold": (("g1_mul", "g2_mul"), sum(K * h for h in hs if K * h > max(fw, FOLD_COMB_MAX))),
        "k_lamc_sum": ("lamc_term", R * M if M <= LAM_COMB_MAX_M else 0),
        "k_msm_chunk": ("msm_madd", 2 * R * M * W if M > LAM_COMB_MAX_M else 0),
        "k_msm_chunk_g2": ("g2_msm_madd", 4 * 2 * R * K * W2 if w_msm else 0),
        "k_w_comb": ("w_comb_term", K * (2 * R - 2) if not w_msm and R <= G2_COMB_MAX_R else 0),
        "k_w_terms": ("g2_mul", w_terms if K * 2 * R > lim["wterm_warp_max"] else 0),
        "k_w_terms_w": ("g2_mul", w_terms if K * 2 * R <= lim["wterm_warp_max"] else 0),
        "k_pst_terms": ("g1_mul", M * lc // 2),
    }


def roofline_report(prof: dict, units: dict, peak: float, t_lane: float, t_split: float, steps: int,
                    log_n: int, b: int, total_ms: float) -> dict:
    """The rooflines of one run from its per-kernel CUDA-event totals `prof` (name -> (launches, ms)
    over `steps` timed steps): the dominant kernel and every kernel with a unit count against the
    multiply-add peak `peak` (lane ops/s), and every round-structured kernel against its latency
    bound (critical product rounds x the measured latency of one dependent product, `t_lane` on one
    lane and `t_split` split over a block's four warps, in ns)."""

    def kernel_roof(kname, cnt, kms):
        if kname not in units or kms <= 0 or units[kname][1] <= 0:
            return None
        unit, n_units = units[kname]
        per_unit = sum(FQ_MULS[u] for u in (unit if isinstance(unit, tuple) else (unit,)))
        ops_step = n_units * per_unit * FQ_MUL_IMAD
        launches_per_step = cnt / steps
        avg_ms = kms / cnt
        achieved = ops_step / launches_per_step / (avg_ms * 1e-3)
        return {"achieved": achieved / 1e12, "frac": achieved / peak, "units_per_step": n_units, "unit_op": unit,
                "launches_per_step": launches_per_step, "avg_launch_ms": avg_ms}

    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("", (0, 0.0))
    name, (cnt, kms) = dom
    roof = None
    r = kernel_roof(name, cnt, kms)
    if r:
        roof = {"bound": "alu", "kernel": name, "achieved": r["achieved"], "peak": peak / 1e12,
                "unit": "Tops/s (32-bit multiply-add lane ops)", "frac": r["frac"],
                "traffic": NCU_TRAFFIC.get((log_n, b, name)),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture of this kernel"
                                  if (log_n, b, name) in NCU_TRAFFIC else None,
                "units_per_step": r["units_per_step"], "unit_op": r["unit_op"],
                "launches_per_step": r["launches_per_step"], "avg_launch_ms": r["avg_launch_ms"],
                "peak_source": "measured: fp_imad_probe on this GPU in this run"}
    roof_all = {}
    for kname, (kc, kt) in prof.items():
        r = kernel_roof(kname, kc, kt)
        if r:
            roof_all[kname] = {"frac": round(r["frac"], 4), "avg_launch_ms": round(r["avg_launch_ms"], 4),
                               "units_per_step": r["units_per_step"], "unit_op": r["unit_op"]}
    # latency bound of every round-structured kernel: rounds x the measured latency of one dependent
    # product (one lane; for the split rounds, the block's four warps together); the headline is the
    # round chain's kernel with the most time per step
    lat_all = {}
    for kname, (kc, kt) in prof.items():
        if kname in CRITICAL_ROUNDS and kc and kt > 0:
            rounds = CRITICAL_ROUNDS[kname]
            sr = SPLIT_ROUNDS.get(kname, 0)
            bound_ms = ((rounds - sr) * t_lane + sr * t_split) * 1e-6
            lat_all[kname] = {"critical_rounds": rounds, "split_rounds": sr, "bound_ms": round(bound_ms, 4),
                              "achieved_ms": round(kt / kc, 4), "frac": round(bound_ms / (kt / kc), 4),
                              "on_round_chain": kname in CHAIN_KERNELS, "ms_per_step": round(kt / steps, 3)}
    lat = None
    chain = [k for k in lat_all if lat_all[k]["on_round_chain"]]
    if chain:
        top = max(chain, key=lambda k: lat_all[k]["ms_per_step"])
        lat = dict(kernel=top, **lat_all[top], fq_mul_ns=t_lane, fq_mul_split_ns=t_split,
                   note="sequential Fq-product rounds of the round chain's largest kernel x the measured "
                        "latency of one dependent product (one lane, or split over a block's four warps for "
                        "the split rounds); combines and inversions excluded; every such kernel in "
                        "latency_rooflines")
    share = {k: round(v[1] / (total_ms if total_ms else 1), 4) for k, v in
             sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]}
    # every kernel: launches per step and mean CUDA-event time per launch (ms)
    kernel_ms = {k: [round(v[0] / steps, 2), round(v[1] / v[0], 4)] for k, v in
                 sorted(prof.items(), key=lambda kv: -kv[1][1]) if v[0]}
    return {"roofline": roof, "roofline_kernels": roof_all, "latency_roofline": lat, "latency_rooflines": lat_all,
            "kernel_share": share, "kernel_launches_and_ms": kernel_ms}


class ClockSampler:
    """nvidia-smi clocks during the timed region (median SM clock, throttle reasons seen)."""

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--log-n", type=int, default=16)
    ap.add_argument("--b", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the N=2^20 b sweep and the MSM sweep")
    ap.add_argument("--fc-only", action="store_true", help="only the FC microbenchmark (one JSON line)")
    ap.add_argument("--msm-sweep", default="12,14,16,18,20,22,24", help="log2 sizes of the MSM sweep")
    ap.add_argument("--b-sweep", default="1,16,256,1024", help="b values of the N=2^20 ProveAll sweep")
    ap.add_argument("--served-requests", type=int, default=100, help="requests of the served trace replayed")
    ap.add_argument("--served-rate", type=float, default=200.0, help="offered rate of the served trace (req/s)")
    ap.add_argument("--served-only", action="store_true",
                    help="only the served workload: the trace at --served-rate (served and sequential) and the "
                         "rate sweep (one JSON line)")
    ap.add_argument("--served-rates", default="2,4,6,8,12,16", help="offered rates of the served rate sweep")
    ap.add_argument("--sweep-requests", type=int, default=150, help="requests per point of the rate sweep")
    ap.add_argument("--batched-only", action="store_true", help="only the 64-job batched workload (one JSON line)")
    ap.add_argument("--schedule", default="direct", choices=["direct", "lookahead"],
                    help="Step-1 round schedule (fp_set_schedule)")
    ap.add_argument("--msm-only", type=int, default=0, metavar="LOG_N",
                    help="time only the standalone G1 MSM of 2^LOG_N points (profiling runs)")
    return ap.parse_args()


def time_device(fn, stream, steps: int, warmup: int, flush=None) -> float:
    """Average ms of fn() on `stream` by CUDA events, after warm-up; L2 flushed before each run."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def proveall_sweep(F, I, torch, np, stream, flush, b_values, seed: int) -> dict:
    """ProveAll (Commit + OpenAll) proofs/s at N = 2^20 for each b (3 warm-up, 3 timed steps)."""
    log_n = 20
    pp = F.PP(log_n, 1, seed, stream)
    m_dev = torch.from_numpy(I.vector(seed + 1, log_n).view(np.int64).copy()).cuda()
    out = {}
    for b in b_values:
        keep = []

        def step():
            cm = F.Commitment(pp, m_dev, stream)
            keep.append((cm, F.Proofs(pp, cm, b, stream)))
            if len(keep) > 2:
                keep.pop(0)
        ms = time_device(step, stream, 3, 3, flush)
        out[f"b={b}"] = {"proofs_per_s": (1 << log_n) / (ms * 1e-3), "ms_per_step": ms}
    return out


def verify_sweep(F, I, torch, np, cases, seed: int) -> dict:
    """vc_verify_all: every proof of one ProveAll output verified against the claimed values
    (device-resident), host wall time of the synchronous call, median of 3 after one warm-up."""
    out = {}
    for log_n, b in cases:
        pp = F.PP(log_n, 1, seed)
        m = I.vector(seed + 1, log_n)
        cm = F.Commitment(pp, m)
        C, _ = cm.get()
        pf = F.Proofs(pp, cm, b)
        md = torch.from_numpy(m.view(np.int64).copy()).cuda()
        torch.cuda.synchronize()
        F.vc_verify_all(pf, C, md)
        ts, n = [], 0
        for _ in range(3):
            t0 = time.perf_counter()
            _, n = F.vc_verify_all(pf, C, md)
            ts.append(time.perf_counter() - t0)
        s = sorted(ts)[1]
        out[f"n2^{log_n}_b={b}"] = {"proofs_per_s": pp.N / s, "ms": s * 1e3, "accepted": n, "N": pp.N}
        del pf, cm, pp
    return out


def fc_microbench(F, I, torch, np, seed: int) -> dict:
    """The FC scheme alone (Table tb:fc and the batch-opening/verification figures), as OpenAll for
    sub-arrays on a split with R = n segments of M = 2 elements: FC.Commit = VC.Commit (two-term
    row MSMs, then the n-pair FC commitment), FC.BOpen-t = Step 1 on one block of t segments,
    t x FC.BOpen-1 = t blocks of one segment (one batched call, and t single calls), FC.BVerify-t =
    the segment verifier on a block of t.  Device time (CUDA events) for Commit and BOpen, host
    wall time for the synchronous verifier (FC.BVerify-t against t calls of FC.BVerify-1 on t
    segments at n = 2^12, the batch-verification figure); median of 3 after one warm-up."""
    s = torch.cuda.Stream()

    def dev_ms(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sorted(ts)[1]

    def wall_ms(fn):
        fn()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            ts.append((time.perf_counter() - t0) * 1e3)
        return sorted(ts)[1]

    out = {"table": {}, "batch_open_n2^12": {}, "batch_verify_n2^12": {}}
    for log_r in (8, 9, 10, 11, 12):
        pp = F.PP(log_r + 1, 1, seed, s, log_r=log_r)
        m = I.vector(seed + 1, log_r + 1)
        m_dev = torch.from_numpy(m.view(np.int64).copy()).cuda()
        keep = []

        def commit():
            keep.append(F.Commitment(pp, m_dev, s))
            if len(keep) > 2:
                keep.pop(0)
        row = {"commit_ms": dev_ms(commit)}
        cm = F.Commitment(pp, m_dev, s)
        C, _ = cm.get(rows=False)
        for t in (1, 32):
            hold = []

            def bopen():
                hold.append(F.vc_open_segments(pp, cm, t, 0, 1, s))
                if len(hold) > 2:
                    hold.pop(0)
            row[f"bopen_t{t}_ms"] = dev_ms(bopen)
            seg = F.vc_open_segments(pp, cm, t, 0, 1, s)
            proof = seg.segment_proof(0)
            assert F.vc_verify_segment(pp, C, t, 0, m[0:2], proof, s)
            row[f"bverify_t{t}_ms"] = wall_ms(lambda: F.vc_verify_segment(pp, C, t, 0, m[0:2], proof, s))
        row["pi_y_bytes"] = 1344 * log_r + 480
        out["table"][f"n=2^{log_r}"] = row
        if log_r == 12:
            one = row["bopen_t1_ms"]
            ones = F.vc_open_segments(pp, cm, 1, 0, 512, s)       # FC.BOpen-1 of segments 0 .. 511
            proofs1 = [ones.segment_proof(j) for j in range(512)]
            for t in (16, 32, 64, 128, 256, 512):
                blk = F.vc_open_segments(pp, cm, t, 0, 1, s).segment_proof(0)
                assert F.vc_verify_segment(pp, C, t, 0, m[0:2], blk, s)

                t0 = time.perf_counter()                            # t calls, timed once
                for j in range(t):
                    assert F.vc_verify_segment(pp, C, 1, j, m[2 * j:2 * j + 2], proofs1[j], s)
                out["batch_verify_n2^12"][f"t={t}"] = {
                    "bverify_t_ms": wall_ms(lambda: F.vc_verify_segment(pp, C, t, 0, m[0:2], blk, s)),
                    "t_x_bverify1_ms": (time.perf_counter() - t0) * 1e3,
                }
            for t in (16, 32, 64, 128, 256, 512):
                hold = []

                def batch_t():
                    hold.append(F.vc_open_segments(pp, cm, t, 0, 1, s))
                    if len(hold) > 2:
                        hold.pop(0)

                def t_single():
                    hold.append(F.vc_open_segments(pp, cm, 1, 0, t, s))
                    if len(hold) > 2:
                        hold.pop(0)
                out["batch_open_n2^12"][f"t={t}"] = {
                    "bopen_t_ms": dev_ms(batch_t),
                    "t_x_bopen1_one_call_ms": dev_ms(t_single),
                    "t_x_bopen1_sequential_ms": t * one,
                }
        del cm, pp
    return out


def eval_sweep(F, I, torch, np, cases, seed: int) -> dict:
    """Evaluation proof of the committed vector's multilinear extension at a random point (prover and
    GPU verifier, host wall time of the synchronous calls, median of 3 after one warm-up)."""
    import random
    out = {}
    for log_n in cases:
        pp = F.PP(log_n, 1, seed)
        m = I.vector(seed + 1, log_n)
        cm = F.Commitment(pp, m)
        C, _ = cm.get(rows=False)
        rnd = random.Random(seed + log_n)
        r = [rnd.randrange(I.R_INT) for _ in range(log_n)]

        def wall(fn):
            fn()
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                fn()
                ts.append((time.perf_counter() - t0) * 1e3)
            return sorted(ts)[1]
        proof = F.vc_eval_prove(pp, cm, r)
        assert F.vc_eval_verify(pp, C, r, proof)
        out[f"n2^{log_n}"] = {"prove_ms": wall(lambda: F.vc_eval_prove(pp, cm, r)),
                              "verify_ms": wall(lambda: F.vc_eval_verify(pp, C, r, proof)),
                              "proof_bytes": len(proof)}
        del cm, pp
    return out


def batched_workload(F, I, torch, np, tune_passes: int = 1) -> dict:
    """64 jobs, log N uniform in 8..18 by seed, b = min(R, nearestpow2(log^2 N)), one SRS for 2^18
    resident: one vc_prove_all_batch captured as a CUDA graph vs the same jobs as concurrent job
    streams vs 64 sequential vc_prove_all calls.  Commitments are made beforehand (not timed)."""
    spec = I.batched_jobs(4, 64, 8, 18)
    parent = F.PP(18, 1, 4)
    views, cms = {}, []
    for sp in spec:
        ln = sp["log_n"]
        if ln not in views:
            views[ln] = parent.view(ln)
        cms.append(F.Commitment(views[ln], I.vector(sp["seed"], ln)))
    jobs = [(cm, sp["b"]) for cm, sp in zip(cms, spec)]
    total = sum(cm.pp.N for cm, _ in jobs)
    s = torch.cuda.current_stream()

    def run(fn, reps, warm):
        for _ in range(warm):
            r = fn()
            torch.cuda.synchronize()
            del r
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            del r
        return min(ts)
    phases = []

    def graph_call():
        r = F.vc_prove_all_batch(jobs, use_graph=True, stream=s)
        phases.append(F.batch_last_times())
        return r
    t_graph = run(graph_call, 3, 2)
    ph = min(phases[-3:], key=lambda p: p["capture_ms"] + p["instantiate_ms"] + p["run_ms"])
    t_streams = run(lambda: F.vc_prove_all_batch(jobs, use_graph=False, stream=s), 3, 1)
    t_seq = run(lambda: [F.Proofs(cm.pp, cm, b, s) for cm, b in jobs], 1, 1)
    # the schedule autotuner on this job mix (engine-choice limits), then the graph again with its choice
    from paper_2601_03031_gb300 import autotune as A
    key = A.batch_key([(sp["log_n"], sp["b"]) for sp in spec])
    t0 = time.perf_counter()
    entry = A.tune_engines(key, lambda: F.vc_prove_all_batch(jobs, use_graph=True, stream=s), reps=2,
                           max_passes=tune_passes)
    tune_s = time.perf_counter() - t0
    phases.clear()
    t_tuned = run(graph_call, 3, 1)
    ph_t = min(phases[-3:], key=lambda p: p["capture_ms"] + p["instantiate_ms"] + p["run_ms"])
    t_seq_tuned = run(lambda: [F.Proofs(cm.pp, cm, b, s) for cm, b in jobs], 1, 1)
    F.set_engine_limits(None)
    return {"jobs": 64, "log_n": sorted(sp["log_n"] for sp in spec), "total_proofs": total,
            "timing": "host wall clock around the call, after synchronize, best of runs",
            "graph": {"ms": t_graph * 1e3, "proofs_per_s": total / t_graph, "phases_ms": ph,
                      "proofs_per_s_graph_run_only": total / (ph["run_ms"] * 1e-3) if ph["run_ms"] else None},
            "graph_tuned": {"ms": t_tuned * 1e3, "proofs_per_s": total / t_tuned, "phases_ms": ph_t,
                            "proofs_per_s_graph_run_only": total / (ph_t["run_ms"] * 1e-3) if ph_t["run_ms"] else None,
                            "limits": entry["limits"], "tuning_s": tune_s, "tuning_trials": len(entry["trials"]),
                            "sequential_same_limits_ms": t_seq_tuned * 1e3},
            "streams": {"ms": t_streams * 1e3, "proofs_per_s": total / t_streams},
            "sequential": {"ms": t_seq * 1e3, "proofs_per_s": total / t_seq}}


def _pct(a, q):
    a = sorted(a)
    return a[min(len(a) - 1, int(q * len(a)))] if a else None


def _served_run(F, I, torch, np, S, trace, vecs, check_solo: int = 0) -> dict:
    """Replay `trace` in real time through the continuous-batching server; latency = arrival to
    proof state in host memory.  The sustained load is completed requests / (last completion -
    first arrival); the backlog is the number of requests waiting or running when the last one
    arrives."""
    srv = S.Server(log_n_max=20, seed=0, slots=32)
    for ln in range(10, 21):
        srv.view(ln)
    for b in (1, 16):
        srv.submit(I.vector(1, 10), b).result()
    t0 = time.perf_counter()
    futs = []
    for r, m in zip(trace, vecs):
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        futs.append(srv.submit(m, r["b"], t_arrival=t0 + r["t"]))
    t_last = t0 + trace[-1]["t"]
    res = [f.result() for f in futs]
    peak = srv.peak_running
    srv.close()
    span = max(q.t_done for q in res) - t0
    backlog = sum(1 for q in res if q.t_done > t_last)
    lat = [q.latency for q in res]
    half = len(res) // 2
    out = {"requests": len(res), "offered_req_per_s": len(res) / max(trace[-1]["t"], 1e-9),
           "sustained_req_per_s": len(res) / span, "span_s": span,
           "proofs_per_s": sum(1 << r["log_n"] for r in trace) / span,
           "p50_ms": _pct(lat, 0.5) * 1e3, "p99_ms": _pct(lat, 0.99) * 1e3,
           "second_half_p50_ms": _pct(lat[half:], 0.5) * 1e3,
           "backlog_at_last_arrival": backlog, "peak_concurrent_jobs": peak}
    if check_solo:
        for q in range(0, len(res), max(1, len(res) // check_solo)):
            r = trace[q]
            C, rows, state = S.solo(srv.view(r["log_n"]), vecs[q], r["b"])
            assert state == res[q].state and C == res[q].C, "served result differs from its solo run"
    return out


def _sequential_run(F, I, torch, np, S, srv_views, trace, vecs) -> dict:
    """The same trace through plain synchronous calls, one request at a time in arrival order
    (vc_commit, vc_prove_all, the proof state copied to the host), replayed in real time."""
    t0 = time.perf_counter()
    lat, t_end = [], t0
    for r, m in zip(trace, vecs):
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        S.solo(srv_views[r["log_n"]], m, r["b"])
        t_end = time.perf_counter()
        lat.append(t_end - (t0 + r["t"]))
    span = t_end - t0
    return {"requests": len(trace), "sustained_req_per_s": len(trace) / span, "span_s": span,
            "proofs_per_s": sum(1 << r["log_n"] for r in trace) / span,
            "p50_ms": _pct(lat, 0.5) * 1e3, "p99_ms": _pct(lat, 0.99) * 1e3}


def served_workload(F, I, torch, np, nreq: int, rate: float = 200.0, sequential: bool = True) -> dict:
    """Poisson trace (seed 5, log N uniform 10..20, b uniform {1, 16, 256} clamped to R) at `rate`
    requests/s, its first nreq requests replayed in real time through the serving loop, and (when
    `sequential`) through plain synchronous calls one at a time, also in real time."""
    from paper_2601_03031_gb300 import serve as S
    trace = I.poisson_trace(5, 2000, rate, 10, 20, (1, 16, 256))[:nreq]
    vecs = [I.vector(r["seed"], r["log_n"]) for r in trace]
    out = {"trace": f"poisson seed 5, {rate:g} req/s, log N 10..20, b in {{1,16,256}}",
           "latency": "arrival to proof state in host memory",
           "served": _served_run(F, I, torch, np, S, trace, vecs, check_solo=10)}
    if sequential:
        views = {}
        base = F.PP(20, 1, 0)
        for ln in range(10, 21):
            views[ln] = base if ln == 20 else base.view(ln)
        out["sequential"] = _sequential_run(F, I, torch, np, S, views, trace, vecs)
    return out


def served_rate_sweep(F, I, torch, np, nreq: int, rates) -> dict:
    """The served trace's request mix at several offered rates (same sizes, seeds and order; arrival
    times from the Poisson stream at each rate): the highest rate whose sustained load keeps up with
    the offered load (within 10 %) and whose backlog at the last arrival stays within the 32 slots."""
    from paper_2601_03031_gb300 import serve as S
    out, best = {}, None
    for rate in rates:
        trace = I.poisson_trace(5, 2000, rate, 10, 20, (1, 16, 256))[:nreq]
        vecs = [I.vector(r["seed"], r["log_n"]) for r in trace]
        r = _served_run(F, I, torch, np, S, trace, vecs)
        r["bounded"] = r["sustained_req_per_s"] >= 0.9 * r["offered_req_per_s"] and r["backlog_at_last_arrival"] <= 32
        out[f"{rate:g}_req_per_s"] = r
        if r["bounded"]:
            best = rate
    out["highest_bounded_rate_req_per_s"] = best
    return out


def msm_sweep(F, I, torch, np, stream, flush, logs, seed: int) -> dict:
    """Standalone G1 MSM, uniform 255-bit scalars, window by the autotuner: Mpts/s per size."""
    out = {}
    for lg in logs:
        n = 1 << lg
        s_dev = torch.from_numpy(I.fr_uniform(seed + 1000 + lg, n).view(np.int64)).cuda()
        k_dev = torch.from_numpy(I.fr_uniform(seed + 2000 + lg, n).view(np.int64)).cuda()
        bases = F.G1Bases(scalars=s_dev, stream=stream)
        res = torch.zeros(96, dtype=torch.uint8, device="cuda")
        window, _ = F.msm_autotune(bases, k_dev, 1, stream)
        ms = time_device(lambda: F.msm_g1(bases, k_dev, 1, 0, stream, res), stream, 5, 3, flush)
        out[f"2^{lg}"] = {"mpts_per_s": n / (ms * 1e-3) / 1e6, "ms": ms, "window": window}
        del bases, s_dev, k_dev
        torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------------------------- oracle arm
def oracle_sample(log_n: int, b: int, seed: int, other_rows: bool = False, threads: int | None = None):
    """Time the CPU oracle, as it stands, on a bounded sample of one Commit + OpenAll step, on
    `threads` host threads (default: every core); return (sample seconds, estimated seconds of the
    full step on the same threads, description, per-part seconds).

    Sample: Commit's row MSMs and Miller loops on one row per thread at once (scaled to R rows),
    the final exponentiation, FC.BOpen on min(K, threads) blocks at once (scaled to all K =
    ceil(R/b) blocks; the oracle runs one block on one thread), and Step 2 in full (one thread).  The
    oracle's rows for the sample come from its own trapdoor closed form, which it knows from its
    setup."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from paper_2601_03031_gb300 import inputs as I

    threads = threads or os.cpu_count() or 1
    r_mod = I.R_INT

    def mle_eval(table, tau):       # f(tau) for the multilinear extension, x_s <-> bit s
        vals = list(table)
        for s in range(len(tau)):
            t = tau[s]
            vals = [(vals[2 * c] + (vals[2 * c + 1] - vals[2 * c]) * t) % r_mod for c in range(len(vals) // 2)]
        return vals[0]

    pp = O.PP(log_n, seed)
    m = I.vector(seed + 1, log_n)
    vals = I.to_ints(m)
    R, M = pp.R, pp.M
    K = (R + b - 1) // b
    beta, tau = pp.trapdoor()
    # rows by closed form (not timed), exactly what the oracle commit produces
    g1 = O.g1_gen()
    fj = [mle_eval(vals[j * M:(j + 1) * M], tau) for j in range(R)]
    rows = b"".join(O.g1_mul(g1, f) for f in fj)
    s = sum(fj[j] * pow(beta, 2 * j, r_mod) for j in range(R)) % r_mod
    C = O.fq12_pow(O.pairing(g1, O.g2_gen()), s)
    lam_top = pp.to_bytes()[96 * (M - 1): 96 * (2 * M - 1)]
    v0 = pp.to_bytes()[96 * (2 * M): 96 * (2 * M) + 192]
    t, scale = {}, {}
    srows = min(R, threads)
    nblk = min(K, threads)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda j: O.g1_msm(lam_top, vals[j * M:(j + 1) * M]), range(srows)))
        t["commit_msm"], scale["commit_msm"] = time.perf_counter() - t0, R / srows
        t0 = time.perf_counter()
        fs = list(ex.map(lambda j: O.miller(rows[96 * j:96 * j + 96], v0), range(srows)))
        t["commit_miller"], scale["commit_miller"] = time.perf_counter() - t0, R / srows
        t0 = time.perf_counter()
        O.final_exp(fs[0])
        t["commit_final_exp"], scale["commit_final_exp"] = time.perf_counter() - t0, 1.0
        t0 = time.perf_counter()
        list(ex.map(lambda k: O.bopen(pp, C, rows, b, k), range(nblk)))
        t["step1"], scale["step1"] = time.perf_counter() - t0, K / nblk
    pr = O.Prover(pp, m.tobytes(), C, rows, b)
    t0 = time.perf_counter()
    pr.step2()
    t["step2"], scale["step2"] = time.perf_counter() - t0, 1.0
    sample_s = sum(t.values())
    full_s = sum(t[k] * scale[k] for k in t)
    desc = (f"N=2^{log_n}, b={b} on {threads} host threads: commit MSM and Miller loops timed on {srows}/{R} rows "
            f"(one per thread, scaled x{R / srows:g}) + 1 final exp; FC.BOpen timed on {nblk} of {K} blocks "
            f"(one per thread, scaled x{K / nblk:g}); Step 2 in full on one thread; {sample_s:.1f} s of sampled "
            f"work per step, full step estimated at {full_s:.1f} s")
    if not other_rows:
        return sample_s, full_s, desc, t
    # the other rows, timed on the same kind of sample (not part of the step total)
    other = {}
    pr.block(0)
    proof = pr.proof(0)
    t0 = time.perf_counter()
    assert O.verify(pp, C, b, 0, vals[0], proof, memo=False)
    other["verify_one_proof_s"] = time.perf_counter() - t0
    import random
    rnd = random.Random(seed + log_n)
    pt = [rnd.randrange(r_mod) for _ in range(log_n)]
    t0 = time.perf_counter()
    ep = O.eval_prove(pp, m.tobytes(), C, rows, pt)
    other["eval_prove_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    assert O.eval_verify(pp, C, pt, ep)
    other["eval_verify_s"] = time.perf_counter() - t0
    # FC alone at n = 2^8 (R = 256 segments of 2), one block of t = 1
    fpp = O.PP(9, seed, log_r=8)
    fbeta, ftau = fpp.trapdoor()
    fvals = I.to_ints(I.vector(seed + 1, 9))
    ffj = [mle_eval(fvals[2 * j:2 * j + 2], ftau) for j in range(256)]
    frows = b"".join(O.g1_mul(g1, f) for f in ffj)
    fs = sum(ffj[j] * pow(fbeta, 2 * j, r_mod) for j in range(256)) % r_mod
    fC = O.fq12_pow(O.pairing(g1, O.g2_gen()), fs)
    t0 = time.perf_counter()
    fproof, _ = O.bopen(fpp, fC, frows, 1, 0)
    other["fc_bopen_n2^8_t1_s"] = time.perf_counter() - t0
    seg = frows[0:96] + fproof
    mj = I.vector(seed + 1, 9)[0:2].tobytes()
    t0 = time.perf_counter()
    assert O.verify_segment(fpp, fC, 1, 0, mj, seg)
    other["fc_bverify_n2^8_t1_s"] = time.perf_counter() - t0
    t["other_rows"] = other
    return sample_s, full_s, desc, t


def fc_oracle_table(seed: int, threads: int | None = None) -> dict:
    """The CPU oracle's FC scheme alone (Table tb:fc) on the same R = n, M = 2 splits as the GPU rows:
    FC.Commit (the oracle's VC.Commit on the split), FC.BOpen-1 and FC.BVerify-1 for n = 2^8 .. 2^10,
    FC.BOpen-32 and FC.BVerify-32 at n = 2^8; each call single-threaded and timed on its own thread,
    the calls spread over the host cores.  n = 2^11, 2^12 are not run (FC.BOpen is linear in n)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from paper_2601_03031_gb300 import inputs as I

    threads = threads or os.cpu_count() or 1
    cases = {}
    for log_r in (8, 9, 10):
        fpp = O.PP(log_r + 1, seed, log_r=log_r)
        mb = I.vector(seed + 1, log_r + 1).tobytes()
        cases[log_r] = (fpp, mb)

    def timed(fn):
        t0 = time.perf_counter()
        r = fn()
        return time.perf_counter() - t0, r

    def row(log_r):
        fpp, mb = cases[log_r]
        out = {}
        out["commit_s"], (C, rows) = timed(lambda: O.commit(fpp, mb))
        for t in ((1, 32) if log_r == 8 else (1,)):
            out[f"bopen_t{t}_s"], (proof, _) = timed(lambda: O.bopen(fpp, C, rows, t, 0))
            seg = rows[0:96 * t] + proof
            out[f"bverify_t{t}_s"], ok = timed(lambda: O.verify_segment(fpp, C, t, 0, mb[0:64], seg))
            assert ok
        return log_r, out

    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = dict(ex.map(row, (8, 9, 10)))
    return {f"n=2^{k}": v for k, v in sorted(res.items())} | {
        "note": "oracle as it stands, one thread per call; n = 2^11, 2^12 not run"}


def run_reference(args):
    """The oracle as it stands on the host cores: each step is one bounded sample of the step
    (oracle_sample); ms_per_step is the sample's own wall time and value the full-step rate the
    sample estimates (N / estimated full-step seconds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.lib()
    N = 1 << args.log_n
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        pass      # the oracle has no warm-up effects worth a sample; warm-up steps are not re-run
    samples, fulls = [], []
    desc = ""
    for _ in range(max(1, args.steps)):
        sample_s, full_s, desc, _parts = oracle_sample(args.log_n, args.b, args.seed, threads=threads)
        samples.append(sample_s)
        fulls.append(full_s)
    value = N / (sum(fulls) / len(fulls))
    ms = 1e3 * sum(samples) / len(samples)
    line = {
        "impl": "reference", "metric": "ProveAll proofs/s (Commit + OpenAll)", "value": value,
        "unit": "proofs/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 limbs (exact Fq/Fr arithmetic)", "data": "synthetic",
        "config": {"workload": f"ProveAll N=2^{args.log_n} b={args.b} uniform Fr, BLS12-381", "log_n": args.log_n,
                   "b": args.b, "step": "one bounded sample of the Commit + OpenAll step (see cpu_baseline.sample)"},
        "cpu_baseline": {"value": value, "unit": "proofs/s", "cores": threads, "kind": "oracle", "sample": desc,
                         "estimated_full_step_s": sum(fulls) / len(fulls)},
        "e2e": {"value": value, "unit": "proofs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------- replicas (N > 1)
def replica_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s vector: every replica proves its own vector."""
    return seed + 1 + rank


def slowest_rank_ms(total_ms: float, world: int, dist=None, device="cpu") -> float:
    """The timed region's length over all ranks (max): the job ends with its slowest replica."""
    if world <= 1:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_proofs_per_s(world: int, N: int, ms_per_step: float) -> float:
    """Whole-job throughput: all ranks' proofs per step over the slowest rank's step time."""
    return world * N / (ms_per_step * 1e-3)


# --------------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2601_03031_gb300 import _lib as F
    from paper_2601_03031_gb300 import inputs as I
    F.set_schedule(args.schedule)

    if args.fc_only:
        res = fc_microbench(F, I, torch, np, args.seed)
        if rank == 0:
            line = {"metric": "FC.BOpen ms (Table tb:fc)", "n_gpus": world, "fc_microbench": res}
            if not args.no_cpu_baseline:
                line["fc_oracle"] = fc_oracle_table(args.seed)
            print(json.dumps(line))
        return
    if args.batched_only:
        res = batched_workload(F, I, torch, np, tune_passes=2)
        if rank == 0:
            print(json.dumps({"metric": "batched ProveAll proofs/s", "value": res["graph_tuned"]["proofs_per_s"],
                              "unit": "proofs/s", "n_gpus": world,
                              "config": {"workload": "64 ProveAll jobs, log N uniform 8..18 (seed 4), b = min(R, "
                                                     "nearest power of two to log^2 N), one SRS for 2^18"},
                              "batched_64_jobs": res}))
        return
    if args.served_only:
        res = served_workload(F, I, torch, np, args.served_requests, args.served_rate)
        sweep = served_rate_sweep(F, I, torch, np, args.sweep_requests,
                                  [float(x) for x in args.served_rates.split(",") if x])
        if rank == 0:
            print(json.dumps({"metric": "served p50/p99 latency and proofs/s", "n_gpus": world,
                              "config": {"workload": f"served Poisson trace, first {args.served_requests} requests "
                                                     f"at {args.served_rate:g} req/s; rate sweep of "
                                                     f"{args.sweep_requests} requests per rate"},
                              "served_trace": res, "rate_sweep": sweep}))
        return
    if args.msm_only:
        stream = torch.cuda.current_stream()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        res = msm_sweep(F, I, torch, np, stream, flush, [args.msm_only], args.seed)
        if rank == 0:
            (k, v), = res.items()
            print(json.dumps({"metric": "MSM Mpts/s", "value": v["mpts_per_s"], "unit": "Mpts/s", "n_gpus": world,
                              "config": {"workload": f"G1 MSM {k} points, uniform Fr scalars", "window": v["window"]},
                              "ms": v["ms"]}))
        return

    log_n, b = args.log_n, args.b
    N = 1 << log_n
    stream = torch.cuda.current_stream()
    pp = F.PP(log_n, b, args.seed, stream)
    m = I.vector(replica_seed(args.seed, rank), log_n)
    m_dev = torch.from_numpy(m.view(np.int64).copy()).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # > 129 MB L2

    def step(mid=None):
        cm = F.Commitment(pp, m_dev, stream)
        if mid is not None:
            mid.record(stream)
        pf = F.Proofs(pp, cm, b, stream)
        return cm, pf

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = F.launch_count()
    F.profile_enable(True)
    F.profile_report()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    keep = []
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            keep.append(step(mids[s]))
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    F.profile_enable(False)
    prof = F.profile_report()
    launches = (F.launch_count() - launches0) / max(1, args.steps)
    total_ms = sum(a.elapsed_time(b_) for a, b_ in ev)
    commit_ms = sum(a.elapsed_time(mid) for (a, _), mid in zip(ev, mids)) / args.steps
    openall_ms = sum(mid.elapsed_time(b_) for (_, b_), mid in zip(ev, mids)) / args.steps
    total_ms = slowest_rank_ms(total_ms, world, dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_proofs_per_s(world, N, ms_per_step)

    # end-to-end through the C ABI with host buffers: H2D of m from pinned memory inside vc_commit,
    # D2H of the shared proof state (the OpenAll result) into pinned memory
    m_host = torch.from_numpy(m.view(np.int64).copy()).pin_memory()
    cm, pf = step()
    state = torch.empty(pf.state_size(), dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cm = F.Commitment(pp, m_host.numpy().view(np.uint64), stream)
        pf = F.Proofs(pp, cm, b, stream)
        pf.state_into(state)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_t) / len(e2e_t)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # rooflines: the dominant kernel against the multiply-add pipe, every kernel with a unit count, and
    # the latency bound of every round-structured kernel
    units = step_units(log_n, b, F.msm_window(pp.M, pp.R), F.msm_window_g2(2 * pp.R, -(-pp.R // b)))
    rep = roofline_report(prof, units, F.imad_peak(), F.fq_mul_latency_ns(), F.fq_mul_split_latency_ns(),
                          args.steps, log_n, b, total_ms)
    roof, roof_all, lat, lat_all = rep["roofline"], rep["roofline_kernels"], rep["latency_roofline"], \
        rep["latency_rooflines"]
    share, kernel_ms = rep["kernel_share"], rep["kernel_launches_and_ms"]

    cpu = None
    if not args.no_cpu_baseline:
        try:
            threads = os.cpu_count() or 1
            sample_s, cpu_s, desc, parts = oracle_sample(log_n, b, args.seed, other_rows=True, threads=threads)
            cpu = {"value": N / cpu_s, "unit": "proofs/s", "cores": threads, "kind": "oracle", "sample": desc,
                   "sample_s": sample_s, "estimated_full_step_s": cpu_s,
                   "other_rows": dict(parts.get("other_rows", {}),
                                      note="one thread each: VC.Verify of one proof (N = 2^%d, b = %d, no "
                                           "sharing), the evaluation proof at a random point (prove, verify), "
                                           "FC.BOpen-1 and FC.BVerify-1 at n = 2^8" % (log_n, b))}
        except Exception as e:      # the baseline is reported, not required for the GPU number
            cpu = {"value": None, "unit": "proofs/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    sweeps = None
    if not args.no_sweeps:
        sweeps = {
            "proveall_n2^20": proveall_sweep(F, I, torch, np, stream, flush,
                                             [int(x) for x in args.b_sweep.split(",") if x], args.seed),
            "msm_g1": msm_sweep(F, I, torch, np, stream, flush,
                                [int(x) for x in args.msm_sweep.split(",") if x], args.seed),
            "verify_all": verify_sweep(F, I, torch, np, [(16, 256), (20, 1), (20, 1024)], args.seed),
            "fc_microbench": fc_microbench(F, I, torch, np, args.seed),
            "eval_proof": eval_sweep(F, I, torch, np, [16, 20], args.seed),
            "batched_64_jobs": batched_workload(F, I, torch, np),
            "served": served_workload(F, I, torch, np, args.served_requests, args.served_rate),
        }

    line = {
        "metric": "ProveAll proofs/s (Commit + OpenAll)", "value": value, "unit": "proofs/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 limbs (exact Fq/Fr arithmetic)", "data": "synthetic",
        "config": {"workload": f"ProveAll N=2^{log_n} b={b} uniform Fr, BLS12-381", "log_n": log_n, "b": b,
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before every timed step",
                   "step1_schedule": args.schedule},
        "e2e": {"value": N / e2e_s, "unit": "proofs/s", "h2d_bytes_per_step": N * 32,
                "d2h_bytes_per_step": int(state.numel())},
        "phases": {"commit_ms": commit_ms, "openall_ms": openall_ms,
                   "openall_only_proofs_per_s": N / (openall_ms * 1e-3),
                   "note": "value counts Commit + OpenAll per step; OpenAll alone is the paper's ProveAll time"},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_kernels": roof_all,
        "latency_roofline": lat,
        "latency_rooflines": lat_all,
        "kernel_share": share,
        "kernel_launches_and_ms": kernel_ms,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "sweeps": sweeps,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
