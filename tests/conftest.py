import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def mpslcc():
    """The GB300 library package, built in-tree if needed."""
    from paper_1509_00216_gb300 import _build
    _build.build()
    import paper_1509_00216_gb300 as m
    return m
