"""Test configuration: the ``gpu`` marker selects tests that need a GB300
and the CUDA library; ``slow`` marks long oracle runs (opt in with
--runslow)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    parser.addoption("--runslow", action="store_true", default=False, help="run long oracle pins")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libhgks")
    config.addinivalue_line("markers", "slow: long CPU oracle run (enable with --runslow)")


def pytest_collection_modifyitems(config, items):
    if config.getoption("--runslow"):
        return
    skip = pytest.mark.skip(reason="slow oracle pin: pass --runslow")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)
