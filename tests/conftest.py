import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size workload checks")


@pytest.fixture(scope="session")
def eo():
    """The CUDA library's Python binding (GPU tests only)."""
    import paper_1806_01036_gb300 as eo_mod
    return eo_mod


@pytest.fixture(scope="session")
def ctx(eo):
    c = eo.Context(0)
    yield c
    c.close()
