import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# keep the schedule-tuning cache of the tests out of the user's cache
os.environ.setdefault("CPC_TUNE_CACHE", os.path.join(ROOT, "_build_test_tune_cache.json"))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-side oracle runs")
