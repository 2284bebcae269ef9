import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libedp.so")


@pytest.fixture(scope="session")
def edp_lib():
    """The CUDA library, built in-tree; GPU tests fail (not skip) without it."""
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_1410_7922_gb300 import build
    build.build()
    from paper_1410_7922_gb300 import edp
    edp.load()
    return edp
