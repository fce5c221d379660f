import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libxs.so")


@pytest.fixture(autouse=True)
def _bounds_checked_status(request):
    """Under XS_CHECKED=1 the GPU tests run on the bounds-checked library; after each
    test no index check may have failed."""
    yield
    if os.environ.get("XS_CHECKED") == "1" and request.node.get_closest_marker("gpu") is not None:
        from paper_2105_14782_gb300 import xs
        if xs._lib is not None:
            assert xs.check_status(clear=True) == 0, "a bounds check failed in the checked build"
