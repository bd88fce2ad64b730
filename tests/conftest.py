import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def rng():
    import numpy as np
    return np.random.default_rng(12345)


@pytest.fixture(scope="session")
def hisq():
    """The CUDA library, built in-tree if stale. Fails (no fallback) when it cannot be built or loaded."""
    import torch
    from paper_2111_10354_gb300 import build
    build.build()
    import paper_2111_10354_gb300 as h
    h.lib()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return h
