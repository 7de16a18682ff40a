import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running statistical check")


def pytest_collection_modifyitems(config, items):
    # tests marked gpu are skipped here only when no GPU is visible and the run
    # did not ask for them explicitly; `-m gpu` on a GPU machine runs them.
    pass
