import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running check")


@pytest.fixture(scope="session")
def small_corpus():
    from paper_2108_00895_gb300 import workloads
    w = workloads.SMALL
    return w, w.corpus(), w.init_ids()
