import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def cuda():
    """The CUDA device with the library built; fails (never skips) when a GPU
    test runs without a GPU or without the library."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0912_3678_gb300 import build
    build.build()
    import paper_0912_3678_gb300 as bt
    bt.load_library()
    return torch.device("cuda:0")


def to_dev(a, device):
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)


def to_host(t):
    return t.detach().cpu().numpy()
