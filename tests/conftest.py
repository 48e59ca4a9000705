import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libkirin")
    config.addinivalue_line("markers", "slow: takes tens of seconds of CPU time")


@pytest.fixture(scope="session")
def kirin_lib():
    """The CUDA library through its C ABI; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0707_0438_gb300 import abi
    return abi.lib()
