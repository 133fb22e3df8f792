import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built liblatms.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def cuda():
    """The GPU tests run only where CUDA exists; they never fall back to the CPU."""
    import torch
    assert torch.cuda.is_available(), "gpu-marked test needs CUDA"
    from paper_1605_05712_gb300 import lib
    lib()  # raises if the native library is missing
    return torch.device("cuda:0")
