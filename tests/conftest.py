import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running full-size case")


@pytest.fixture(scope="session")
def hooks_lib():
    """The test build of the library (libgbfft_testhooks.so): the same kernels
    as libgbfft.so, plus environment overrides of planner choices (passes,
    splits, staging kernels, tile sizes) and the fault switch of the
    bounded-wait test.  Tests that force a planner choice through the
    environment run on this build; the product library ignores the variables."""
    from paper_1707_07263_gb300 import _lib, build_lib
    return _lib.load(build_lib.TEST_LIB)
