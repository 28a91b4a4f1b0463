import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-side oracle runs")


@pytest.fixture(scope="session")
def coupling_cache():
    from oracle import sh

    cache = {}

    def get(N):
        if N not in cache:
            mats = sh.coupling(N)
            cache[N] = (mats, sh.placement(N, mats))
        return cache[N]

    return get
