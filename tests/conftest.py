import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # gpu tests are skipped (not failed) on a machine without a GPU when run unfiltered
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture
def gemm_cluster():
    """Sets the CTAs per cluster of the LSC tensor-core GEMMs for one test (1 or 2) and
    restores each GEMM's default afterwards."""
    from paper_1808_01517_gb300 import _lib as L

    yield L.set_gemm_cluster
    L.set_gemm_cluster(0)
