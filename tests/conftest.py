import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def rs():
    """The CUDA library's Python binding, built in-tree for sm_103a."""
    import paper_1301_4019_gb300 as rs_mod
    rs_mod.load()
    return rs_mod


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
