import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run on the GB300 box)")


@pytest.fixture(scope="session")
def h2mech():
    from paper_2508_16105_gb300 import synth
    return synth.h2_air_mechanism(16105)


@pytest.fixture(scope="session")
def h2oracle(h2mech):
    import oracle
    return oracle.Oracle(h2mech.to_text())
