"""GPU deflation set-up (sgn_build_deflation) against the dense eigendecomposition.

The eigenvalues of smallest |lambda| are unique; the eigenvectors carry a free
phase, so the comparison is on the phase-invariant projector P = R L^dag and on
the properties L^dag R = I and A R = R Lambda."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _check(dims, U, mu, A, m, extra, dec=None):
    import paper_0910_2927_gb300 as pkg
    R0, L0, lam0, nxt0 = O.critical_eigenpairs(A, m, extra=extra, decomposition=dec)
    with pkg.SignContext(dims, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        lam = ctx.build_deflation(m, extra=extra, eig_tol=1e-10)
        R, L, lamd = ctx.get_deflation()
    np.testing.assert_allclose(lam[:m], lam0, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(lam[m:], nxt0, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(lamd, lam0, rtol=1e-9)
    assert np.abs(L.conj().T @ R - np.eye(m)).max() < 1e-9
    # eigen-residuals through the oracle's operator
    AR = np.stack([O.hw(dims, U, R[:, j], mu) for j in range(m)], axis=1)
    rel = np.linalg.norm(AR - R * lamd, axis=0) / (np.abs(lamd) * np.linalg.norm(R, axis=0))
    assert rel.max() < 1e-9
    # same oblique projector as the dense eigenvectors
    P, P0 = R @ L.conj().T, R0 @ L0.conj().T
    assert np.abs(P - P0).max() < 1e-7 * np.abs(P0).max()


def test_small_lattice():
    dims, mu = (3, 2, 3, 4), 0.3
    U = si.random_su3_links(dims, 0.7, 21)
    A = O.dense_hw(dims, U, mu)
    _check(dims, U, mu, A, 6, 2)


def test_config1_lattice(lattice4):
    d = lattice4
    _check(d["dims"], d["U"], d["mu"], d["A"], 8, 4, dec=d["eig"])


def test_mu0_hermitian():
    dims = (3, 3, 2, 4)
    U = si.random_su3_links(dims, 0.7, 31)
    A = O.dense_hw(dims, U, 0.0)
    _check(dims, U, 0.0, A, 5, 3)
