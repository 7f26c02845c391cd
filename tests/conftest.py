"""Shared pytest configuration: the ``gpu`` marker and repo-root imports."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def gpu():
    """The built CUDA library and a context on cuda:0 (gpu tests only; fails without a GPU)."""
    import torch
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    from paper_2003_01836_gb300 import build
    build.build()
    import paper_2003_01836_gb300 as b
    ctx = b.Context(0)
    yield ctx
    ctx.close()
