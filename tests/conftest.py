"""Shared pytest set-up: the ``gpu`` marker and the repository root on ``sys.path``."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test (still part of the CPU suite)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def ba():
    """The CUDA library's Python binding (built first; fails loudly when CUDA is missing)."""
    import torch

    from paper_1602_07106_gb300 import build as ba_build
    ba_build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1602_07106_gb300 import ba as module
    return module
