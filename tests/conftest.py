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


@pytest.fixture(scope="session")
def rtpn_lib():
    """The built library (built in-tree on first use)."""
    from paper_2004_02833_gb300 import build, rtpn

    build.build()
    return rtpn.lib()


def _cuda_ok():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda_device(rtpn_lib):
    if not _cuda_ok():
        pytest.fail("a CUDA device is required for gpu-marked tests")
    import torch

    torch.cuda.init()
    return torch.device("cuda:0")
