"""Stored expected values (tests/golden/, written by make_golden.py from the oracle)."""
import os

import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    return np.loadtxt(os.path.join(HERE, name), comments="#")


def test_kenney_laub_table_closed_form():
    """eq. (6.2) at s = 4: the stored table equals the trigonometric closed form."""
    t = _load("kenney_laub_s4.txt")
    th = np.pi * (np.arange(1, 5) - 0.5) / 8
    np.testing.assert_allclose(t[:, 0], -np.tan(th) ** 2, rtol=1e-15)
    np.testing.assert_allclose(t[:, 1], 1 / (4 * np.cos(th) ** 2), rtol=1e-15)


def test_oracle_reproduces_stored_solution():
    g = _load("fomlr_2x2x3x2.txt")
    x_ref = g[:, 0] + 1j * g[:, 1]
    dims = (2, 2, 3, 2)
    U = si.random_su3_links(dims, 0.7, 77)
    b = si.gaussian_field(dims, 78)
    sigma, omega = O.kenney_laub(8, 0.5)
    x, rep, _ = O.fom_lr(dims, U, b, 0.3, sigma, omega, k=12, tol=1e-13, max_cycles=5000)
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


@pytest.mark.gpu
def test_gpu_matches_stored_solution():
    torch = pytest.importorskip("torch")
    import paper_0910_2927_gb300 as pkg
    g = _load("fomlr_2x2x3x2.txt")
    x_ref = g[:, 0] + 1j * g[:, 1]
    dims = (2, 2, 3, 2)
    U = si.random_su3_links(dims, 0.7, 77)
    b = si.gaussian_field(dims, 78)
    sigma, omega = pkg.kenney_laub(8, 0.5)
    with pkg.SignContext(dims, mu=0.3) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=12, tol=1e-13, max_cycles=5000)
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
    x = x.cpu().numpy()
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
