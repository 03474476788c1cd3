import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~10 s")


@pytest.fixture(scope="session")
def psl7():
    """The seeded PSL(2,7), Delta=6 instance and its oracle code (index 0 of seed 0)."""
    import workloads
    from oracle import tanner
    inst = workloads.standard("PSL(2,7)", 0)
    return inst, tanner.from_instance(inst)


@pytest.fixture(scope="session")
def sl3():
    """The seeded SL(2,3), Delta=4 instance and its oracle code (index 0 of seed 0)."""
    import workloads
    from oracle import tanner
    inst = workloads.standard("SL(2,3)", 0)
    return inst, tanner.from_instance(inst)
