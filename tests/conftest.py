import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def lattice16():
    from paper_2511_21921_gb300 import synth
    return synth.load("lattice16")


@pytest.fixture(scope="session")
def lognormal32():
    from paper_2511_21921_gb300 import synth
    return synth.load("lognormal32")
