import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfsl.so")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def fsl():
    """The CUDA library binding; builds libfsl.so if it is missing or stale."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2207_14496_gb300 import build
    build.build()
    from paper_2207_14496_gb300 import fsl as mod
    return mod
