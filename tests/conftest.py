import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # Keep the file named test_zz_* last whatever the selection order.
    items.sort(key=lambda it: 1 if os.path.basename(str(it.fspath)).startswith("test_zz_") else 0)


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_runtest_setup(item):
    if item.get_closest_marker("gpu") is not None and not _cuda_available():
        if os.environ.get("GRES_REQUIRE_GPU"):
            pytest.fail("GRES_REQUIRE_GPU is set but no CUDA device is available")
        pytest.skip("no CUDA device")
