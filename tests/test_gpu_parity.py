"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, byte for byte.

There is no floating point anywhere in the method, so the tolerance is zero: public parameters,
commitments and every proof byte must be identical.  Small cases compare everything; the
N = 2^16 and N = 2^20 cases compare all shared Step-2 state and sampled Step-1 blocks / proofs,
and check commitments against the trapdoor closed form.
"""
import functools
import os
import random
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyref as ref
from tests import _pyec, _state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402


@functools.lru_cache(maxsize=None)
def gpu_pp(log_n, seed):
    return F.PP(log_n, 1, seed)


@functools.lru_cache(maxsize=None)
def oracle_pp(log_n, seed):
    return O.PP(log_n, seed)


@functools.lru_cache(maxsize=None)
def vec(log_n, seed, dist="uniform"):
    return I.vector(seed, log_n, dist)


@functools.lru_cache(maxsize=None)
def gpu_commit(log_n, seed, dist="uniform"):
    return F.Commitment(gpu_pp(log_n, seed), vec(log_n, seed + 1, dist))


@functools.lru_cache(maxsize=None)
def oracle_commit(log_n, seed, dist="uniform"):
    return O.commit(oracle_pp(log_n, seed), vec(log_n, seed + 1, dist).tobytes())


@pytest.mark.parametrize("log_n", [2, 3, 4, 5, 10])
def test_setup_parity(log_n):
    assert gpu_pp(log_n, 7).export() == oracle_pp(log_n, 7).to_bytes()


@pytest.mark.parametrize("log_n,dist", [(2, "uniform"), (4, "uniform"), (5, "uniform"), (10, "uniform"),
                                        (10, "u32")])
def test_commit_parity(log_n, dist):
    assert gpu_commit(log_n, 7, dist).get() == oracle_commit(log_n, 7, dist)


@pytest.mark.parametrize("log_n,b", [(2, 1), (2, 2), (4, 1), (4, 3), (4, 4), (5, 1), (5, 3), (5, 4)])
def test_prove_all_every_proof(log_n, b, schedule):
    seed = 7
    pp, opp = gpu_pp(log_n, seed), oracle_pp(log_n, seed)
    m = vec(log_n, seed + 1)
    C, rows = oracle_commit(log_n, seed)
    pf = F.Proofs(pp, gpu_commit(log_n, seed), b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    assert pf.step2_parts() == pr.step2_parts()
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r)
    got = pf.export(0, pp.N)
    exp = b"".join(pr.proof(i) for i in range(pp.N))
    assert got == exp
    vals = I.to_ints(m)
    assert all(O.verify_many(opp, C, b, [(i, vals[i], pr.proof(i)) for i in range(pp.N)]))


def test_config1_n1024_b1_all_proofs_and_verify(schedule):
    """N = 2^10, b = 1, seed 0: every one of the 1024 proofs equals the oracle's and verifies."""
    log_n, seed, b = 10, 0, 1
    pp, opp = F.PP(log_n, b, seed), O.PP(log_n, seed)
    m = I.vector(seed, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    pf = F.Proofs(pp, cm, b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r)
    got = pf.export(0, pp.N)
    off = 0
    vals = I.to_ints(m)
    items = []
    for i in range(pp.N):
        e = pr.proof(i)
        assert got[off:off + len(e)] == e, i
        items.append((i, vals[i], e))
        off += len(e)
    assert off == len(got)
    assert all(O.verify_many(opp, C, b, items))


def test_empty_and_degenerate_vectors(schedule):
    """All-zero vector (identity rows, e(O, .) = 1) and a single non-zero entry."""
    log_n, seed, b = 4, 3, 2
    pp, opp = gpu_pp(log_n, seed), oracle_pp(log_n, seed)
    for m in (np.zeros((16, 4), np.uint64), np.eye(1, 16, 9, dtype=np.uint64).reshape(16, 1) * np.array([5, 0, 0, 0], np.uint64)):
        m = np.ascontiguousarray(m, dtype=np.uint64)
        cm = F.Commitment(pp, m)
        C, rows = O.commit(opp, m.tobytes())
        assert cm.get() == (C, rows)
        pf = F.Proofs(pp, cm, b)
        pr = O.Prover(opp, m.tobytes(), C, rows, b)
        pr.blocks(); pr.step2()
        _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r)
        assert pf.export(0, 16) == b"".join(pr.proof(i) for i in range(16))


def test_range_error():
    pp = gpu_pp(4, 7)
    m = np.zeros((16, 4), np.uint64)
    m[3] = np.array(I.R_LIMBS, np.uint64)
    with pytest.raises(F.FlexProofsError) as e:
        F.Commitment(pp, m)
    assert e.value.status == 6


def test_device_input_matches_host_input():
    log_n, seed = 5, 7
    pp = gpu_pp(log_n, seed)
    m = vec(log_n, seed + 1)
    t = torch.from_numpy(m.view(np.int64).copy()).cuda()
    cm = F.Commitment(pp, t, stream=torch.cuda.current_stream())
    assert cm.get() == oracle_commit(log_n, seed)


# ------------------------------------------------------------------ N = 2^16 (benchmark workload)
def row_closed_form(opp, m_ints):
    """(C, rows) from the oracle's trapdoor by the closed form, in pure Python (tests._pyec)."""
    beta, tau = opp.trapdoor()
    return _pyec.commit_closed_form(groups(), beta, tau, opp.R, opp.M, m_ints)


@functools.lru_cache(maxsize=None)
def groups():
    return _pyec.Groups(O.g1_gen(), O.g2_gen())


@functools.lru_cache(maxsize=None)
def n16(dist):
    """GPU commitment of the N = 2^16 vector, and the oracle side's commitment from the trapdoor
    closed form (the oracle's inputs never come from the GPU)."""
    log_n, seed = 16, 0
    pp, opp = gpu_pp(log_n, seed), oracle_pp(log_n, seed)
    m = vec(log_n, seed + 1, dist)
    cm = F.Commitment(pp, m)
    return pp, opp, m, cm, row_closed_form(opp, I.to_ints(m))


@pytest.mark.parametrize("dist", ["uniform", "u32"])
def test_n16_commit_closed_form(dist):
    pp, opp, m, cm, exp = n16(dist)
    assert cm.get() == exp


@pytest.mark.parametrize("b,blocks,dist", [(256, [0], "uniform"), (1, [0, 77, 128, 255], "uniform"),
                                          (256, [0], "u32"), (1, [0, 255], "u32")])
def test_n16_prove_all_sampled(b, blocks, dist, schedule):
    """OpenAll at N = 2^16 in the benchmark's launch configuration: the whole shared state (every
    Merkle digest, r_j, every fold-tree node D_w and g_w, every PST quotient commitment) equal to
    the oracle's, the block records of the oracle's blocks (all of them at b = 256), and sampled
    proofs byte-identical and accepted by the oracle's verifier."""
    pp, opp, m, cm, (C, rows) = n16(dist)
    pf = F.Proofs(pp, cm, b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks(blocks)
    pr.step2()
    assert pf.step2_parts() == pr.step2_parts()
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r, blocks)
    rnd = random.Random(5)
    vals = I.to_ints(m)
    for k in blocks:
        j = k * b + rnd.randrange(min(b, pp.R - k * b))
        for a in (0, rnd.randrange(pp.M), pp.M - 1):
            i = j * pp.M + a
            e = pr.proof(i)
            assert pf.proof(i) == e
            assert O.verify(opp, C, b, i, vals[i], e)


@pytest.mark.parametrize("log_n,b", [(4, 1), (5, 3), (6, 8)])
def test_prove_one_equals_oracle_brute_force_and_prove_all(log_n, b, schedule):
    """vc_prove_one (Step 1 on the index's block only) against the oracle's brute-force
    single-index prover and against vc_prove_all's proof, for every index of a ragged layout."""
    seed = 9
    pp, opp = gpu_pp(log_n, seed), oracle_pp(log_n, seed)
    m = vec(log_n, seed + 1)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    pf = F.Proofs(pp, cm, b)
    for i in range(pp.N):
        one = F.vc_prove_one(pp, cm, b, i)
        assert one == pf.proof(i), i
        if i % 5 == 0:
            assert one == O.prove_one(opp, m.tobytes(), C, rows, b, i), i


def test_prove_one_n16_sampled(schedule):
    pp, opp, m, cm, (C, rows) = n16("uniform")
    vals = I.to_ints(m)
    for b, i in ((256, 12345), (1, 65535), (16, 40000)):
        one = F.vc_prove_one(pp, cm, b, i)
        assert one == O.prove_one(opp, m.tobytes(), C, rows, b, i)
        assert O.verify(opp, C, b, i, vals[i], one)
    with pytest.raises(F.FlexProofsError):
        F.vc_prove_one(pp, cm, 1, pp.N)


# ------------------------------------------------------------------ N = 2^20, b = 1024, 256, 16, 1
# Step-1 blocks compared per b (K = 1, 4, 64, 1024 blocks): every block at b >= 256, eight spread
# over the 64 at b = 16 and 32 spread over the 1024 at b = 1 (first and last included).
N20_BLOCKS = {1024: [0], 256: [0, 1, 2, 3], 16: [9 * i for i in range(8)],
              1: [round(i * 1023 / 31) for i in range(32)]}


@functools.lru_cache(maxsize=None)
def n20():
    log_n, seed = 20, 0
    pp, opp = gpu_pp(log_n, seed), oracle_pp(log_n, seed)
    m = vec(log_n, seed + 1)
    return pp, opp, m, F.Commitment(pp, m), row_closed_form(opp, I.to_ints(m))


@functools.lru_cache(maxsize=None)
def n20_oracle():
    """Oracle provers for every b: Step 2 in full and Step 1 on the sampled blocks, run on host
    threads (each call releases the GIL; the jobs write disjoint parts of the provers)."""
    pp, opp, m, cm, (C, rows) = n20()
    provers = {b: O.Prover(opp, m.tobytes(), C, rows, b) for b in N20_BLOCKS}
    jobs = [p.step2 for p in provers.values()]
    jobs += [functools.partial(provers[b].block, k) for b, ks in N20_BLOCKS.items() for k in ks]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for f in [ex.submit(j) for j in jobs]:
            f.result()
    return provers


def test_n20_setup_and_commit_closed_form():
    pp, opp, m, cm, exp = n20()
    assert pp.export() == opp.to_bytes()
    assert cm.get() == exp


@pytest.mark.parametrize("b,sched", [(1024, "direct"), (1024, "lookahead"), (256, "direct"), (256, "lookahead"),
                                     (16, "direct"), (1, "direct")])
def test_n20_prove_all_sampled(b, sched):
    """OpenAll at N = 2^20 in the benchmark's launch configuration: Step-2 state equal to the
    oracle's, sampled proofs of the sampled blocks byte-identical and accepted by the oracle's
    verifier, and every one of the 2^20 proofs accepted by the GPU batch verifier."""
    pp, opp, m, cm, (C, rows) = n20()
    pr = n20_oracle()[b]
    F.set_schedule(sched)
    try:
        pf = F.Proofs(pp, cm, b)
    finally:
        F.set_schedule("direct")
    assert pf.step2_parts() == pr.step2_parts()
    _state.assert_equal(pf.state(), pr.state(), pp.R, pp.M, pr.K, opp.log_r, N20_BLOCKS[b])
    rnd = random.Random(b)
    vals = I.to_ints(m)
    items = []
    for k in N20_BLOCKS[b]:
        j = k * b + rnd.randrange(min(b, pp.R - k * b))
        for a in (0, rnd.randrange(pp.M), pp.M - 1):
            i = j * pp.M + a
            e = pr.proof(i)
            assert pf.proof(i) == e, i
            items.append((i, vals[i], e))
    assert all(O.verify_many(opp, C, b, items))
    ok, n_ok = F.vc_verify_all(pf, C, m)
    assert n_ok == pp.N and ok.all()
