import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: large workload")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build_oracle()
    return oracle


# bound every device-side wait and every enumeration run in the tests
os.environ.setdefault("GFD_WAIT_LIMIT_MS", "10000")
os.environ.setdefault("GFD_RUN_LIMIT_MS", "120000")
