import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny_system():
    import synth
    return synth.make_system(2, 2, 1, seed=3)        # 4 atoms: m = 32, n = 8


@pytest.fixture(scope="session")
def small_system():
    import synth
    return synth.make_system(2, 2, 2, seed=1)        # 8 atoms: m = 64, n = 16


@pytest.fixture(scope="session")
def c1_system():
    import synth
    return synth.make_system(4, seed=0)              # 64 atoms: m = 512, n = 128
