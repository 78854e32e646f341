import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ph():
    import phantom
    phantom.build(gpu=False)
    return phantom


@pytest.fixture(autouse=True)
def _checked_build_faults(request):
    """With MCTP_LIBRARY=checked (the bounds-tested library), every GPU test
    ends by reading the kernels' index-fault bits: any bit fails the test."""
    yield
    if os.environ.get("MCTP_LIBRARY") != "checked" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2311_15038_gb300 import _lib
    if _lib._lib is None:
        return
    import ctypes
    bits = ctypes.c_uint32()
    rc = _lib._lib.mctp_checked_status(ctypes.byref(bits), 1)
    assert rc == 0 and bits.value == 0, f"checked build: index fault bits {bits.value:#x} (rc {rc})"
