import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libbcg.so")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its Python binding; built on first use."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_11930_gb300 import bcg
    bcg.load()
    return bcg
