import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfwikkt.so")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle checks")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lib():
    """The in-tree CUDA library (built on demand); GPU tests only."""
    import paper_2204_06489_gb300 as P
    from paper_2204_06489_gb300 import _build
    _build.build()
    return P.load()
