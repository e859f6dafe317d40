import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libsci.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def gpu():
    """The CUDA path, loaded for real: fails (does not skip) when it is unavailable."""
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_18185_gb300 import build, sci

    build.build()
    sci.load()
    return torch
