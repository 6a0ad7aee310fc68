import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def qfdlib():
    """Builds (if stale) and loads libqfd.so; GPU tests use it through the C ABI."""
    from paper_2006_16935_gb300 import build, qfd

    build.build_library()
    return qfd.load()
