import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def k0():
    import math
    return 2.0 * math.pi


@pytest.fixture(scope="session")
def vielib():
    """Build (if stale) and load libvie.so."""
    from paper_2508_16471_gb300 import build
    build.build()
    from paper_2508_16471_gb300 import vie
    return vie
