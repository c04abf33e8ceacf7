import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (runs the CUDA path through the C ABI)")
    config.addinivalue_line("markers", "slow: long oracle run; enabled with CLBM_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("CLBM_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle run (set CLBM_SLOW=1)")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)
