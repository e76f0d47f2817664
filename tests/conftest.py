import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(autouse=True)
def _oracle_on_all_cores(request):
    """GPU tests run the oracle with its per-element loops split over the host's
    cores (Sec. V); the frames are identical to the sequential oracle's
    (tests/test_oracle_threads.py), only sums over the frame add in another
    order.  CPU tests keep the sequential default."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    import oracle
    prev = oracle.set_threads(min(16, os.cpu_count() or 1))
    yield
    oracle.set_threads(prev)
