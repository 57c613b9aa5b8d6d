"""Shared pytest configuration: the ``gpu`` marker and small helpers."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU statistical test")


def gpu_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ianus():
    """The CUDA library binding; GPU tests fail loudly if it cannot load."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_0704_3573_gb300 as pkg

    return pkg
