import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def c0():
    import gen
    return gen.config_c0()


@pytest.fixture(scope="session")
def c0_system(c0):
    from oracle import scf
    return scf.build_system(c0, keep_metric=True)


@pytest.fixture(scope="session")
def c0_scf(c0_system):
    from oracle import scf
    return scf.rhf(c0_system)
