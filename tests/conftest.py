import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU run")


@pytest.fixture(autouse=True)
def _reset_oracle_mutation():
    yield
    try:
        import oracle
        oracle.set_mutation(0)
    except Exception:
        pass
