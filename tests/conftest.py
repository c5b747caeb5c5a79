import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test (minutes)")


@pytest.fixture(scope="session")
def cap_small():
    import oracle
    import synth
    v, f = synth.cap_bowl_mesh(n_rim=30, n_interior=140, seed=0)
    return oracle.mesh(v, f)


@pytest.fixture(scope="session")
def cap_full():
    import oracle
    import synth
    v, f = synth.cap_bowl_mesh()
    return oracle.mesh(v, f)


@pytest.fixture(scope="session")
def cap_full_F(cap_full):
    import numpy as np
    import oracle
    V = oracle.visibility_rows(cap_full, np.arange(cap_full.n))
    return oracle.F_rows(cap_full, np.arange(cap_full.n), V), V
