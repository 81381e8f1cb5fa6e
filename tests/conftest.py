import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: statistical test taking tens of seconds")


@pytest.fixture(scope="session")
def gfk_lib():
    """The CUDA library; GPU tests fail loudly if it cannot be built or loaded."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_1703_08977_gb300 import gfk
    return gfk
