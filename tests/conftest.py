"""Shared fixtures.  GPU tests are marked ``gpu``; everything else runs on CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def wl():
    from paper_2407_14783_b300 import workloads
    return workloads


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library; GPU tests fail loudly (no fallback) if it is missing."""
    from paper_2407_14783_b300 import build, binding
    build.build()
    return binding.lib()


@pytest.fixture
def make_sim(cuda_lib):
    from paper_2407_14783_b300.sim import Sim
    made = []

    def _make(params, **kw):
        s = Sim(params, **kw)
        made.append(s)
        return s

    yield _make
    for s in made:
        s.close()
