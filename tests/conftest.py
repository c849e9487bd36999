import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running oracle comparison")


def pytest_collection_modifyitems(config, items):
    # Keep the no-allocation entry point's test last even when files are reordered.
    items.sort(key=lambda it: 1 if "test_zz_" in it.nodeid else 0)
