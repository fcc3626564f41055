import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes tens of seconds on the CPU")


def pytest_collection_modifyitems(config, items):
    # GPU tests need the CUDA library; fail loudly (not skip) if the GPU is there but the
    # library is not, so a missing build never passes silently.
    pass
