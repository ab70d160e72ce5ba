import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "oracle_fullsize: compares a full-size GPU result with the oracle "
                            "(the oracle runs on a background thread from the end of collection)")


def pytest_collection_finish(session):
    """Start the full-size oracle states early when a test that needs them is
    selected and a GPU is present, so the host cores work while the GPU
    tests run."""
    if not any(item.get_closest_marker("oracle_fullsize") for item in session.items):
        return
    import torch
    if torch.cuda.is_available():
        from tests import fullsize_oracle
        fullsize_oracle.start()


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as O
    O.lib()
    return O


@pytest.fixture(scope="session")
def qvlib():
    """libqv.so (built if stale) through the ctypes binding."""
    from paper_2508_15545_gb300 import build
    build.build()
    from paper_2508_15545_gb300 import qv
    return qv


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="session")
def fullsize_oracle():
    from tests import fullsize_oracle as F
    return F.get()
