import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library loaded through its ctypes binding (GPU tests only)."""
    import paper_2511_01793_gb300 as emg
    emg.load()
    return emg


@pytest.fixture(autouse=True)
def _bounds_check_clean(request):
    """In the bounds-check build (EMG_BUILD_VARIANT=boundscheck) every GPU test
    must leave the kernels' index-check error word clear."""
    yield
    if os.environ.get("EMG_BUILD_VARIANT") == "boundscheck" and request.node.get_closest_marker("gpu"):
        import paper_2511_01793_gb300 as emg

        assert emg.emg_debug_bounds_errors() == 0
