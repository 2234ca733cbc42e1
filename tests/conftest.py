import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def gspm_lib():
    """Build (if stale) and load libgspm.so; the binding raises if it is missing."""
    from paper_2510_09812_gb300 import build
    build.build()
    from paper_2510_09812_gb300 import gspm
    return gspm
