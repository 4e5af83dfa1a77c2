import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs of more than a few seconds")


@pytest.fixture(scope="session")
def small_params():
    from paper_2602_15104_gb300 import workload as W
    return W.SMALL_TT.params()[0]
