import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


@pytest.fixture(params=["direct", "lookahead"])
def schedule(request):
    """Runs a GPU test under each Step-1 round schedule (the proofs must not depend on it)."""
    from paper_2601_03031_gb300 import _lib as F
    F.set_schedule(request.param)
    yield request.param
    F.set_schedule("direct")
