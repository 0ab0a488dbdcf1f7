import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libbssn.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(autouse=True)
def _no_out_of_range_access(request):
    """Under BSSN_BOUNDS_CHECK=1 the GPU tests run on the bounds-check build
    of the library (libbssn_check.so): after each one, no kernel may have
    recorded an access outside its arrays."""
    yield
    if os.environ.get("BSSN_BOUNDS_CHECK") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import torch
    if not torch.cuda.is_available():
        return
    from paper_1307_6488_gb300 import binding as B
    status, count = B.bounds_violations()
    assert count == 0 and status == B.OK, f"{count} out-of-range accesses recorded"
