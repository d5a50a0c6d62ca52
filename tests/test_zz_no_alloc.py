"""The allocation-free row-commitment entry point, checked through the C ABI against vc_commit.

vc_commit_rows_noalloc exists for callers that cannot allocate device memory (their allocator owns
the device, or an allocation's implicit synchronisation is not acceptable where they run).  It uses
one static device scratch array shared by all calls, so this test makes two calls in a row with
different vectors and checks that each one equals the allocating entry point's rows exactly (the
method is exact integer arithmetic: zero tolerance).  It is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_03031_gb300 import _lib as F  # noqa: E402
from paper_2601_03031_gb300 import inputs as I  # noqa: E402


def rows_via_commit(pp, m):
    return F.Commitment(pp, m).get()[1]


def rows_via_noalloc(pp, m, stream):
    m_dev = torch.from_numpy(np.ascontiguousarray(m).view(np.int64).copy()).cuda()
    out = torch.zeros(96 * pp.R, dtype=torch.uint8, device="cuda")
    F.vc_commit_rows_noalloc(pp, m_dev, out, stream)
    return bytes(out.cpu().numpy())


@pytest.mark.parametrize("log_n", [4, 10, 14])
def test_noalloc_rows_match_commit_two_calls(log_n):
    pp = F.PP(log_n, 1, 5)
    stream = torch.cuda.current_stream()
    for seed in (21, 22):                      # two calls in a row on the shared scratch
        m = I.vector(seed, log_n)
        assert rows_via_noalloc(pp, m, stream) == rows_via_commit(pp, m)


def test_noalloc_limits_and_range():
    pp_big = F.PP(15, 1, 5)                    # N = 2^15 > 2^14
    m = torch.zeros((1 << 15, 4), dtype=torch.int64, device="cuda")
    out = torch.zeros(96 * pp_big.R, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FlexProofsError) as e:
        F.vc_commit_rows_noalloc(pp_big, m, out)
    assert e.value.status == 1
    pp = F.PP(4, 1, 5)
    bad = np.zeros((16, 4), np.uint64)
    bad[7] = np.array(I.R_LIMBS, np.uint64)
    with pytest.raises(F.FlexProofsError) as e:
        rows_via_noalloc(pp, bad, None)
    assert e.value.status == 6
    good = I.vector(3, 4)                      # the status word is cleared by the next call
    assert rows_via_noalloc(pp, good, None) == rows_via_commit(pp, good)


def test_noalloc_allocates_no_device_memory():
    """The device's free memory is the same before and after further calls (inputs, outputs and
    torch's caching allocator all set up beforehand; the first call did the one-time set-up)."""
    log_n = 14
    pp = F.PP(log_n, 1, 5)
    stream = torch.cuda.current_stream()
    m_dev = torch.from_numpy(np.ascontiguousarray(I.vector(31, log_n)).view(np.int64).copy()).cuda()
    out = torch.zeros(96 * pp.R, dtype=torch.uint8, device="cuda")
    F.vc_commit_rows_noalloc(pp, m_dev, out, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        F.vc_commit_rows_noalloc(pp, m_dev, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
