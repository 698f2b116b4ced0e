import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu():
    """The built library on a CUDA device (GPU tests fail loudly without one)."""
    import torch
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_2501_07535_gb300 import build, moma
    build.build()
    moma.lib()
    torch.cuda.init()
    return moma
