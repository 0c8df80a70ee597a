import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def tiny():
    """A 3x3 mesh with a 32-triangle sphere: every dense statement fits."""
    import oracle
    import workloads
    p = workloads.constant(3, 1, 0.5, 1.0, 0.9, 1.0)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=1)
    return p, disc, ops
