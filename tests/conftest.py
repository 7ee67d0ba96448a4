import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads")


@pytest.fixture(scope="session")
def fj():
    """The CUDA library binding (loads libfj.so; fails loudly if missing)."""
    from paper_2301_10841_gb300 import fj as fjmod
    return fjmod


@pytest.fixture(scope="module")
def ctx(fj):
    """A context on cuda:0 for the tests of one module."""
    c = fj.Context(0)
    yield c
    c.close()

