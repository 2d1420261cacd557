import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a); parity tests through the C-ABI")
    config.addinivalue_line(
        "markers", "slow: long-running test (full-size inputs)")


def pytest_collection_modifyitems(config, items):
    # keep the file named test_zz_* last so that a run stopped at the first
    # failure has already run everything else
    items.sort(key=lambda it: os.path.basename(str(it.fspath)).startswith("test_zz_"))
