import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the built CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def bdct_lib():
    """The built CUDA library (built in-tree on first use)."""
    from paper_2609_28519_gb300 import build as B
    B.build()
    from paper_2609_28519_gb300 import native
    return native.lib()


@pytest.fixture(scope="session")
def cuda_dev(bdct_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a host without a CUDA device")
    return torch.device("cuda:0")
