import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libcroft")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def croft_lib():
    """The built C-ABI library loaded through the Python binding (builds it if missing)."""
    from paper_2002_04896_gb300 import build as _build
    _build.ensure_built()
    from paper_2002_04896_gb300 import croft
    return croft
