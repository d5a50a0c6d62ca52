"""vc_verify on the GPU against the oracle's verifier: honest proofs verify, tampered ones do not.

Tampering covers every part of a proof: the claimed value m_i, a block commitment C_a, a GT and a
G1 part of an FC round, the fast-verification proof W, a Merkle path digest, a sibling pair and a
PST proof element; each must be rejected by both verifiers."""
import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402


def setup(log_n, seed, b):
    """GPU proofs, and the oracle's commitment and prover for the same vector: the oracle's
    verifier is only ever handed the oracle's own inputs (equal bytes, asserted)."""
    pp = F.PP(log_n, 1, seed)
    opp = O.PP(log_n, seed)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, rows = O.commit(opp, m.tobytes())
    assert cm.get() == (C, rows)
    pf = F.Proofs(pp, cm, b)
    pr = O.Prover(opp, m.tobytes(), C, rows, b)
    pr.blocks()
    pr.step2()
    return pp, opp, I.to_ints(m), C, pf, pr


@pytest.mark.parametrize("log_n,b", [(4, 1), (5, 3), (6, 8)])
def test_honest_proofs_verify(log_n, b):
    pp, opp, vals, C, pf, pr = setup(log_n, 31, b)
    for i in range(0, pp.N, 3):
        p = pr.proof(i)
        assert pf.proof(i) == p, i
        assert F.vc_verify(pp, C, b, i, vals[i], p), i
        assert O.verify(opp, C, b, i, vals[i], p, memo=False)


def flip(p: bytes, off: int) -> bytes:
    return p[:off] + bytes([p[off] ^ 1]) + p[off + 1:]


def test_tampered_proofs_rejected():
    log_n, b = 5, 2
    pp, opp, vals, C, pf, pr = setup(log_n, 32, b)
    i = 13
    p = pr.proof(i)
    assert pf.proof(i) == p
    nk = b
    lr, lc = pp.log_r, pp.log_c
    fc = 96 * nk
    path = fc + lr * 1344 + 96 + 192 + 192
    sib = path + 32 * (lr + lc)
    pst = sib + 128 * lr
    cases = {
        "m_i": (vals[i] + 1, p),
        "C_a": (vals[i], flip(p, 47)),
        "L_1.T": (vals[i], flip(p, fc + 100)),
        "R_1.1": (vals[i], flip(p, fc + 576 + 96 + 576 + 95)),
        "W": (vals[i], flip(p, path - 1)),
        "path": (vals[i], flip(p, path + 3)),
        "sibling": (vals[i], flip(p, sib + 100)),
        "pst": (vals[i], flip(p, pst + 95)),
    }
    assert F.vc_verify(pp, C, b, i, vals[i], p)
    for name, (mi, q) in cases.items():
        assert not F.vc_verify(pp, C, b, i, mi, q), name
        assert not O.verify(opp, C, b, i, mi, q, memo=False), name
    assert not F.vc_verify(pp, C, b, i, vals[i], p[:-1])          # wrong length
    assert not F.vc_verify(pp, C, b, i + 1, vals[i + 1], p)       # proof of another index
    assert not F.vc_verify(pp, C, b, i, I.R_INT + vals[i], p)     # m_i >= r


def test_verify_n16_sampled():
    log_n, seed = 16, 0
    pp = F.PP(log_n, 1, seed)
    m = I.vector(seed + 1, log_n)
    vals = I.to_ints(m)
    cm = F.Commitment(pp, m)
    C, _ = cm.get()                  # GPU values into the GPU verifier only
    for b, i in ((256, 12345), (1, 65535)):
        pf = F.Proofs(pp, cm, b)
        p = pf.proof(i)
        assert F.vc_verify(pp, C, b, i, vals[i], p)
        assert not F.vc_verify(pp, C, b, i, vals[i] ^ 1, p)


def limbs_of(v: int):
    return [(v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(4)]


@pytest.mark.parametrize("log_n,b", [(4, 1), (5, 3), (7, 4), (10, 1)])
def test_verify_all_matches_single_and_oracle(log_n, b):
    """vc_verify_all over all N proofs: honest values all verify; wrong claimed values (proof 0,
    whose root is the sharing reference, a row-0 proof that is a column's reference, others, and
    a value >= r) fail exactly where vc_verify and the oracle's verifier fail, with and without
    column sharing."""
    import numpy as np
    pp, opp, vals, C, pf, pr = setup(log_n, 41, b)
    N, M = pp.N, pp.M
    m = np.array([limbs_of(v) for v in vals], np.uint64)
    ok, n = F.vc_verify_all(pf, C, m)
    assert n == N and ok.all()
    bad = {0, 1, M + 2, N - 1, N // 2 + 3}
    claimed = list(vals)
    for i in bad:
        claimed[i] = (vals[i] + 1) % I.R_INT
    claimed[N // 2 + 3] = vals[N // 2 + 3] + I.R_INT          # not canonical
    m2 = np.array([limbs_of(v) for v in claimed], np.uint64)
    ok2, n2 = F.vc_verify_all(pf, C, m2)
    assert set(np.nonzero(~ok2)[0].tolist()) == bad and n2 == N - len(bad)
    ok3, n3 = F.vc_verify_all(pf, C, m2, each=True)
    assert (ok3 == ok2).all() and n3 == n2
    for i in sorted(bad | {2, M, N - 2}):
        p = pf.proof(i)
        assert F.vc_verify(pp, C, b, i, claimed[i], p) == ok2[i], i
    for i in (0, 2, N - 1):
        assert pf.proof(i) == pr.proof(i)
        assert O.verify(opp, C, b, i, claimed[i], pr.proof(i), memo=False) == ok2[i], i


def test_verify_all_wrong_commitment_and_device_values():
    import numpy as np
    log_n, b = 6, 2
    pp, opp, vals, C, pf, pr = setup(log_n, 42, b)
    m = np.array([limbs_of(v) for v in vals], np.uint64)
    other = F.Commitment(pp, I.vector(99, log_n))
    C2, _ = other.get()
    ok, n = F.vc_verify_all(pf, C2, m)
    assert n == 0 and not ok.any()
    md = torch.from_numpy(m.view(np.int64)).cuda()
    ok, n = F.vc_verify_all(pf, C, md)
    assert n == pp.N and ok.all()


@pytest.mark.parametrize("b", [256, 1])
def test_verify_all_n16(b):
    """N = 2^16: every proof verifies; two wrong values fail, and only those."""
    import numpy as np
    log_n, seed = 16, 0
    pp = F.PP(log_n, 1, seed)
    m = I.vector(seed + 1, log_n)
    cm = F.Commitment(pp, m)
    C, _ = cm.get()                  # GPU values into the GPU verifier only
    pf = F.Proofs(pp, cm, b)
    ok, n = F.vc_verify_all(pf, C, m)
    assert n == pp.N and ok.all()
    m2 = m.copy()
    m2[777, 0] ^= 1
    m2[65535, 1] ^= 4
    ok2, n2 = F.vc_verify_all(pf, C, m2)
    assert n2 == pp.N - 2 and not ok2[777] and not ok2[65535]
    vals = I.to_ints(m2)
    assert not F.vc_verify(pp, C, b, 777, vals[777], pf.proof(777))
