import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def xf():
    """The C-ABI binding, loaded on a machine with a GPU (fails loudly if the library is missing)."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_1912_10596_gb300 import xflat
    return xflat
