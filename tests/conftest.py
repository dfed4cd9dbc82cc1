import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # run the no-allocation entry point's test file last, whatever the selection
    items.sort(key=lambda it: 1 if os.path.basename(str(it.fspath)).startswith("test_zz") else 0)
