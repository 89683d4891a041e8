import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU check")
    config.addinivalue_line("markers", "widening: a feature beyond the core hot path (tangent augmentation, "
                                       "refinement order); runs after the core tests")


def pytest_collection_modifyitems(session, config, items):
    # core parity first, so that a stopped run (-x) still reports the core
    # path; the allocation-free backward's file stays last
    def rank(it):
        if os.path.basename(str(it.fspath)) == "test_zz_no_alloc.py":
            return 2
        return 1 if it.get_closest_marker("widening") is not None else 0
    items.sort(key=rank)


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle
