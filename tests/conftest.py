import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running check")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(autouse=True)
def _bounds_checks(request):
    # Under the bounds-checked build (TL_DEBUG=1) every GPU test must leave
    # no failed index check behind.
    yield
    if os.environ.get("TL_DEBUG") == "1" and request.node.get_closest_marker("gpu"):
        import torch
        if not torch.cuda.is_available():
            return
        import paper_1804_07250_gb300 as T
        r = T.debug_checks(clear=True)
        assert r["failures"] == 0, "failed bounds checks: %s" % r
