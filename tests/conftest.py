import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs through the C ABI)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def repo_root():
    return ROOT


@pytest.fixture(scope="session")
def hr_oracle():
    """The 4096 x 2560-sample workload (256^3 density) and the FP64 oracle's
    A, R, G on 8192 random targets -- about 2.2e11 FP64 pairs, computed once
    per session and shared by the direct, field and mesh tests."""
    import numpy as np

    import inputs
    import oracle
    p = inputs.make_problem("hr")
    idx = np.sort(np.random.default_rng(4).choice(p.N, size=8192, replace=False))
    A0, R0, G0 = oracle.forces(p.K.astype(np.float64), p.grid, targets=idx)
    return p, idx, A0, R0, G0
