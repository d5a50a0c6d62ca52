"""Engine-choice limits (fp_set_engine_limits) change which kernels run, never the bytes: OpenAll
under the latency engines only, the throughput engines only and mixes of them equals the oracle
(whole state and every proof), and the MSM with other chunk and segment counts equals the naive
per-term MSM of the oracle; the autotuner's table round-trips."""
import json

import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402
from paper_2601_03031_gb300 import autotune as A  # noqa: E402

BIG = 0xFFFFFFFF
PRESETS = {
    "threads": {"miller_block_max": 0, "miller_warp_max": 0, "miller_group_min": 0, "commit_block_max": 0,
                "commit_warp_max": 0, "fe_block_max": 0, "fe_warp_max": 0, "pair_block_max": 0, "fold_warp_max": 0,
                "wterm_warp_max": 0},
    "warps": {"miller_block_max": 0, "miller_warp_max": BIG, "commit_block_max": 0, "commit_warp_max": BIG,
              "fe_block_max": 0, "fe_warp_max": BIG, "pair_block_max": BIG, "fold_warp_max": BIG,
              "wterm_warp_max": BIG},
    "blocks": {"miller_block_max": BIG, "commit_block_max": BIG, "fe_block_max": BIG, "pair_block_max": BIG},
}


@pytest.fixture
def limits():
    yield F.set_engine_limits
    F.set_engine_limits(None)


@pytest.mark.parametrize("preset", sorted(PRESETS))
@pytest.mark.parametrize("log_n,b", [(5, 1), (6, 3)])
def test_openall_equal_under_every_engine(preset, log_n, b, limits):
    seed = 61
    opp = O.PP(log_n, seed)
    m = I.vector(seed + 1, log_n)
    C, rows = O.commit(opp, m.tobytes())
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    limits(PRESETS[preset])
    pp = F.PP(log_n, 1, seed)
    cm = F.Commitment(pp, m)
    assert cm.get() == (C, rows)
    pf = F.Proofs(pp, cm, b)
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r)
    assert pf.export(0, pp.N) == b"".join(pr.proof(i) for i in range(pp.N))


@pytest.mark.parametrize("chunks,segs", [(1, 1), (64, 4), (1 << 20, 1 << 20)])
def test_msm_equal_under_chunk_and_segment_counts(chunks, segs, limits):
    import numpy as np
    rnd = np.random.default_rng(5)
    n = 300
    s = [int(v) % I.R_INT for v in rnd.integers(1, 2**62, n)]
    k = [int(v) for v in rnd.integers(0, 2**62, n)]
    k[7] = I.R_INT - 1
    g = O.g1_gen()
    pts = b"".join(O.g1_mul(g, v) for v in s)
    bases = F.G1Bases(points=pts)
    limbs = np.array([[(v >> (64 * w)) & (2**64 - 1) for w in range(4)] for v in k], np.uint64)
    limits({"msm_chunks": chunks, "msm_segment_threads": segs})
    for window in (0, 5, 11):
        assert F.msm_g1(bases, limbs, 1, window) == O.g1_msm(pts, k)


def test_tuning_table_round_trip(tmp_path):
    path = str(tmp_path / "t.json")
    key = A.batch_key([(8, 16), (9, 16), (8, 16)])
    assert key == "batch:8/16x2;9/16x1"
    A.save_entry(key, {"limits": {"fe_block_max": 0}, "ms": 1.0}, path)
    assert json.load(open(path))[key]["limits"] == {"fe_block_max": 0}
    try:
        assert A.apply(key, path)
        assert F.engine_limits()["fe_block_max"] == 0
        assert not A.apply("absent", path)
    finally:
        F.set_engine_limits(None)
