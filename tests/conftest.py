import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU physics pins (still part of the CPU suite)")


@pytest.fixture(scope="session")
def orc():
    """The CPU oracle module (built on first use)."""
    from oracle import oracle as o
    o.build()
    o.load()
    return o
