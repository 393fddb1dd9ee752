import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def built_lib():
    """Build the C-ABI libraries in-tree if they are missing."""
    from paper_2009_01287_gb300 import binding, build
    if not (os.path.exists(binding.LIB_PATH) and os.path.exists(binding.INSPECT_PATH)):
        build.build()
    return binding


@pytest.fixture(scope="session")
def cuda_device(built_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected but no CUDA device is visible")
    torch.cuda.init()
    return torch.device("cuda:0")
