import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


import pytest


@pytest.fixture(scope="session")
def built_lib():
    """Path of libpowerlu.so, building it (nvcc, sm_103a) when missing."""
    from paper_2002_07138_gb300 import build as _b
    if not os.path.exists(_b.LIB):
        _b.build()
    return _b.LIB


@pytest.fixture(scope="session")
def ctx(built_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    import paper_2002_07138_gb300 as plu
    c = plu.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()
