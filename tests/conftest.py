import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU and the built CUDA library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def ps():
    """The ctypes binding of libps.so (built in-tree on first use)."""
    from paper_1705_08210_gb300 import build_lib
    build_lib.build()
    from paper_1705_08210_gb300 import ps as _ps
    return _ps


@pytest.fixture(scope="session")
def handle(ps):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    h = ps.Handle(0)
    yield h
    h.close()
