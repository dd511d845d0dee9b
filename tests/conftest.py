import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle check")


@pytest.fixture(scope="session")
def cuda_device():
    """The GPU tests run only where a CUDA device is visible; there the CUDA
    library must load (a missing library is an error, not a skip)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    from paper_2502_20610_gb300 import fdtd
    fdtd.load_library()  # raises if the built library is missing
    return torch.device("cuda:0")
