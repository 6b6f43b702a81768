import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def oracle_bin():
    """Builds the C oracles once and returns a path lookup."""
    from oracle import build as ob
    ob.build()
    return ob.binary


@pytest.fixture(scope="session")
def gf_lib():
    """The built runtime library loaded through its binding (GPU tests only)."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2306_11686_gb300 import gf
    return gf
