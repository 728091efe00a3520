import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libgpulsm.so")
    config.addinivalue_line("markers", "slow: large inputs (minutes)")


@pytest.fixture(scope="session")
def lsm_lib():
    """The compiled C-ABI library, built once per session."""
    import __graft_entry__ as g
    g.build()
    from paper_1707_05354_gb300 import gpulsm
    return gpulsm
