"""Shared fixtures.

``-m "not gpu"`` tests run anywhere (oracle pins, generators, host logic, ABI symbols).
``-m gpu`` tests need a CUDA device; they skip when torch sees none, and fail loudly when a
device is present but the CUDA library cannot be built or loaded.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _cuda_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device visible to torch")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def lb():
    """The CUDA library's Python binding (built in-tree on first use)."""
    from paper_2212_08964_gb300 import lbspmv

    lbspmv.ensure_loaded()
    return lbspmv


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
