import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running check")


@pytest.fixture(scope="session")
def tiny():
    import synthetic
    return synthetic.make_system("tiny")


@pytest.fixture(scope="session")
def tiny_soft():
    import synthetic
    return synthetic.make_system("tiny", soft=True)


@pytest.fixture(scope="session")
def tiny_oracle(tiny):
    import oracle
    return oracle.Oracle(tiny)


@pytest.fixture(scope="session")
def soft_oracle(tiny_soft):
    import oracle
    return oracle.Oracle(tiny_soft)
