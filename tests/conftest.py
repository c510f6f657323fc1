import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs the kernels through the C ABI")


def _has_cuda() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_cuda():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def mtb_lib():
    """The CUDA library, built in-tree (nvcc cross-compiles without a GPU)."""
    from paper_2007_06483_gb300 import build

    build.build()
    import paper_2007_06483_gb300 as mtb

    mtb.lib()
    return mtb


@pytest.fixture(params=["auto", "staged", "items"])
def search_kernel(request, monkeypatch):
    """The shift search has two kernels, the staged cluster kernel and the item
    kernel.  The library picks one by stack size and call mode, and
    MTB_SEARCH_ITEMS (read at every launch) forces one: 0 the staged kernel, 1
    the item kernel.  The parity tests run under the library's choice and under
    each kernel forced."""
    if request.param == "staged":
        monkeypatch.setenv("MTB_SEARCH_ITEMS", "0")
    elif request.param == "items":
        monkeypatch.setenv("MTB_SEARCH_ITEMS", "1")
    else:
        monkeypatch.delenv("MTB_SEARCH_ITEMS", raising=False)
    return request.param
