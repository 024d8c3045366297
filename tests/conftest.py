"""Shared pytest configuration: the `gpu` marker and session-scoped fixtures."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def lattice4():
    """4^4 lattice, spread 0.5, mu = 0.3: the small plain-FP64 workload.

    Dense operator, its 8 + 4 critical eigenpairs, and a Gaussian source."""
    import seeded_inputs as si
    import oracle as O
    dims = (4, 4, 4, 4)
    g_seed, b_seed, c_seed = si.CONFIG_SEEDS[1]
    U = si.random_su3_links(dims, 0.5, g_seed)
    A = O.dense_hw(dims, U, 0.3)
    dec = O.eig(A)
    R, L, lam, nxt = O.critical_eigenpairs(A, 8, extra=4, decomposition=dec)
    b = si.gaussian_field(dims, b_seed)
    return dict(dims=dims, U=U, A=A, R=R, L=L, lam=lam, lam_next=nxt, b=b, mu=0.3, eig=dec)
