import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libcoro")
    config.addinivalue_line("markers", "slow: oracle cases that take more than a few seconds")


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library through its Python binding, on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06467_gb300 import coro
    return coro.Library.get()
