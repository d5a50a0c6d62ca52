"""bench.py's roofline accounting on the CPU: the units each kernel processes per step add up to the
operation counts of the protocol (FC.Commit: R Miller loops and one final exponentiation; FC.BOpen
per block: 2(R - 1) Miller loops, 2 log R final exponentiations, R - 1 G1 and R - 1 G2 fold
multiplications, Sec. 3's efficiency analysis; the W proof's 2R - 2 terms per block, Sec. 3 "Faster
verification"; the commit's N terms, Sec. 4.1), whichever engine a round's size selects, and every
unit has an Fq-multiplication count."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# the library's default engine limits as its header documents them (checked against the library below)
DEFAULT_LIMITS = {"miller_block_max": 1024, "miller_warp_max": 16383, "miller_group_min": 1 << 18,
                  "commit_block_max": 1024, "commit_warp_max": 16384, "fe_block_max": 256,
                  "fe_warp_max": (1 << 32) - 1, "pair_block_max": 2048, "fold_warp_max": 4096,
                  "wterm_warp_max": 4096, "msm_chunks": 1 << 17, "msm_segment_threads": 1 << 15}
# settings that move every size boundary, so that each engine's branch is taken somewhere
OTHER_LIMITS = dict(DEFAULT_LIMITS, miller_block_max=8, miller_warp_max=64, miller_group_min=128,
                    commit_block_max=4, commit_warp_max=16, fe_block_max=2, fe_warp_max=8,
                    fold_warp_max=2, wterm_warp_max=8)

CONFIGS = [(log_n, b) for log_n in (4, 8, 10, 16, 20) for b in (1, 4, 16, 256, 1024)
           if b <= 1 << (log_n // 2)]


def units(u, kinds):
    return sum(n for unit, n in u.values() if (unit if isinstance(unit, tuple) else (unit,))[0] in kinds)


def test_documented_defaults_are_the_librarys():
    try:
        from paper_2601_03031_gb300 import _lib as F
        lib = F.default_engine_limits()
    except Exception as e:                      # the library not built in this checkout
        pytest.skip(f"library not loadable: {e}")
    assert lib == DEFAULT_LIMITS


@pytest.mark.parametrize("lim", [DEFAULT_LIMITS, OTHER_LIMITS], ids=["default", "moved"])
@pytest.mark.parametrize("log_n,b", CONFIGS)
def test_units_sum_to_the_protocol_counts(log_n, b, lim):
    lr = log_n // 2
    R, M = 1 << lr, 1 << (log_n - lr)
    K = -(-R // b)
    u = bench.step_units(log_n, b, 16, lim=lim)
    # Miller loops: Commit's R plus 2(R - 1) per block (the multi-pair engine counts pairs)
    assert units(u, {"miller_loop", "miller_loop_multi4"}) == R + K * 2 * (R - 1)
    # final exponentiations: Commit's one plus 2 log R per block
    assert units(u, {"final_exp"}) == 1 + 2 * K * lr
    # fold multiplications: R - 1 points of A and of v per block, by combs or by scalar multiplication
    folds = sum(n for k, (unit, n) in u.items() if k in ("k_fold_c", "k_fold_w", "k_fold"))
    assert folds == K * (R - 1)
    # the comb chains and tables serve exactly the comb folds
    assert u["k_comb_chain"][1] == u["k_fold_c"][1] == u["k_comb_tab"][1]
    # W terms: 2R - 2 per block, by exactly one of the three paths
    w = [u[k][1] for k in ("k_w_comb", "k_w_terms", "k_w_terms_w")]
    g2msm = u["k_msm_chunk_g2"][1]
    assert (sum(w) == K * (2 * R - 2) and g2msm == 0) or (sum(w) == 0 and g2msm > 0)
    # commit: N comb terms or the Pippenger MSM, never both
    assert (u["k_lamc_sum"][1] == R * M) != (u["k_msm_chunk"][1] > 0)
    # sparse G1 terms: the support of b in every round
    assert u["k_sparse_g"][1] == sum(K * min(b, 2 * (R >> j)) for j in range(1, lr + 1))


@pytest.mark.parametrize("log_n,b", CONFIGS)
def test_every_unit_has_a_product_count(log_n, b):
    for kernel, (unit, n) in bench.step_units(log_n, b, 16, lim=DEFAULT_LIMITS).items():
        for x in unit if isinstance(unit, tuple) else (unit,):
            assert bench.FQ_MULS[x] > 0, (kernel, x)


def test_roofline_report_from_event_totals():
    """The bench line's rooflines from per-kernel CUDA-event totals: the dominant kernel's fraction is
    its algorithmic multiply-adds per launch over its mean launch time against the peak, and every
    round-structured kernel's latency fraction is its bound over its mean launch time."""
    steps, peak, t_lane, t_split = 10, 12.0e12, 1380.0, 980.0
    # name -> (launches, total ms) over `steps` steps, shaped like an N = 2^16, b = 256 run
    prof = {"k_sparse_g": (80, 113.4), "k_final_exp_c": (90, 78.8), "k_round_miller_c": (80, 62.8),
            "k_fold_c": (80, 15.1), "k_lamc_sum": (10, 12.4), "k_g1_pair": (330, 10.6)}
    units = bench.step_units(16, 256, 16, lim=DEFAULT_LIMITS)
    rep = bench.roofline_report(prof, units, peak, t_lane, t_split, steps, 16, 256, 204.0)
    roof = rep["roofline"]
    assert roof["kernel"] == "k_sparse_g" and roof["bound"] == "alu"
    ops_per_launch = 510 * bench.FQ_MULS["g1_mul"] * bench.FQ_MUL_IMAD / 8
    assert roof["frac"] == pytest.approx(ops_per_launch / (113.4 / 80 * 1e-3) / peak)
    assert roof["traffic"] is None                       # no capture of this kernel on this build
    lam = rep["roofline_kernels"]["k_lamc_sum"]
    assert lam["units_per_step"] == 1 << 16
    assert lam["frac"] == pytest.approx((1 << 16) * 352 * bench.FQ_MUL_IMAD / 1.24e-3 / peak, abs=1e-4)
    assert "k_g1_pair" not in rep["roofline_kernels"]   # no unit count: not a roofline kernel
    lat = rep["latency_roofline"]
    assert lat["kernel"] == "k_final_exp_c"             # the round chain's kernel with the most time
    fe = bench.CRITICAL_ROUNDS["k_final_exp_c"], bench.SPLIT_ROUNDS["k_final_exp_c"]
    bound = ((fe[0] - fe[1]) * t_lane + fe[1] * t_split) * 1e-6
    assert lat["bound_ms"] == pytest.approx(bound, abs=1e-4)
    assert lat["frac"] == pytest.approx(bound / (78.8 / 90), abs=1e-4)
    assert not rep["latency_rooflines"]["k_sparse_g"]["on_round_chain"]
    assert rep["kernel_launches_and_ms"]["k_g1_pair"] == [33.0, round(10.6 / 330, 4)]


@pytest.mark.parametrize("log_n,b", [(4, 1), (4, 4), (5, 2), (6, 8)])
def test_units_match_the_oracles_counted_operations(log_n, b):
    """The same counts against the operations the oracle performs (counted inside it) when it
    commits and opens every block: Miller loops, final exponentiations, G2 multiplications (folds
    of v and the W terms) and the commitment's terms; the GPU's sparse G1 terms are at most the
    oracle's, which folds a dense b."""
    import oracle as O
    from paper_2601_03031_gb300 import inputs as I
    pp = O.PP(log_n, 5)
    m = I.vector(7, log_n).tobytes()
    R = pp.R
    K = -(-R // b)
    O.ops_reset()
    C, rows = O.commit(pp, m)
    for k in range(K):
        O.bopen(pp, C, rows, b, k)
    ops = O.ops()
    u = bench.step_units(log_n, b, 16, lim=DEFAULT_LIMITS)
    assert ops["miller"] == units(u, {"miller_loop", "miller_loop_multi4"})
    assert ops["final_exp"] == units(u, {"final_exp"})
    g2 = sum(n for k, (unit, n) in u.items() if k in ("k_fold_c", "k_fold_w", "k_fold")) + \
        sum(u[k][1] for k in ("k_w_comb", "k_w_terms", "k_w_terms_w"))
    assert ops["g2_mul"] == g2
    folds_g1 = sum(n for k, (unit, n) in u.items() if k in ("k_fold_c", "k_fold_w", "k_fold"))
    commit_terms = u["k_lamc_sum"][1]
    assert commit_terms == pp.R * pp.M
    assert folds_g1 + u["k_sparse_g"][1] <= ops["g1_mul"] - commit_terms
