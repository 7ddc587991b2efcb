import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libmpw.so")
    config.addinivalue_line("markers", "slow: longer oracle runs (still CPU)")


@pytest.fixture(scope="session")
def mpw_lib():
    """The CUDA library, built in-tree on first use."""
    from paper_2002_00088_gb300.build import build_library
    build_library()
    from paper_2002_00088_gb300 import mpw
    return mpw
