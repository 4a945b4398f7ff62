import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _no_wait_timeouts(request):
    """After every GPU test: no large-polygon CTA gave up waiting for a staged tile (such a CTA
    keeps its bits exact by recomputing from global memory, but the event is never expected)."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    from paper_2306_04316_gb300 import _lib
    if _lib._lib is None:
        return
    import torch
    if not torch.cuda.is_available():
        return
    torch.cuda.synchronize()
    from paper_2306_04316_gb300 import api
    assert api.pip_get_stats()["wait_timeouts"] == 0, "a staged-tile wait timed out"
