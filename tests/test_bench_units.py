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
