import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU statistical test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def emc():
    """The CUDA library, built in-tree for sm_103a (no fallback: a missing
    build or device fails the test)."""
    from paper_1707_09073_gb300 import build
    build.build()
    import paper_1707_09073_gb300 as m
    m.lib()
    return m
