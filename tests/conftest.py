import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _sync_after_gpu_test(request):
    """Synchronise after every GPU test so an asynchronous device error is
    reported by the test that caused it."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    try:
        import torch
        if torch.cuda.is_available():
            torch.cuda.synchronize()
    except RuntimeError as e:
        pytest.fail("device error after %s: %s" % (request.node.nodeid, e))
