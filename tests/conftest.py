import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only test")


def pytest_collection_modifyitems(config, items):
    """GPU tests fail loudly when no GPU is present instead of silently passing;
    the CPU-only run deselects them with -m "not gpu"."""
    return None


@pytest.fixture(scope="session")
def lib():
    """The built CUDA library (product path).  Raises if it is missing."""
    from paper_1611_08678_gb300 import abm
    return abm.load()
