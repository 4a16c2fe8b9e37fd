import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def spand_lib():
    """Builds (if needed) and loads libspand.so.  Host-only entry points
    (analysis, queries, argument checks) work without a GPU."""
    import shutil

    from paper_1901_02971_gb300 import build as B
    if not B.up_to_date() and shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build libspand.so")
    B.build()
    from paper_1901_02971_gb300 import _lib
    return _lib.lib()


@pytest.fixture(scope="session")
def cuda_ok(spand_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True
