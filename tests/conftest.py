import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300 / sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # keep the file that must run last at the end regardless of plugin ordering
    last = [it for it in items if os.path.basename(str(it.fspath)).startswith("test_zz_")]
    rest = [it for it in items if it not in last]
    items[:] = rest + last
