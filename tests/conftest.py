import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "manual: minutes of CPU; skipped unless --runmanual")


def pytest_addoption(parser):
    parser.addoption("--runmanual", action="store_true", default=False,
                     help="also run tests marked manual (minutes of CPU)")


def pytest_collection_modifyitems(config, items):
    if config.getoption("--runmanual"):
        return
    import pytest
    skip = pytest.mark.skip(reason="manual: run with --runmanual")
    for item in items:
        if "manual" in item.keywords:
            item.add_marker(skip)
