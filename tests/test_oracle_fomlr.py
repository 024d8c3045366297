"""Pins for the oracle's restarted FOM-LR(m,k) (Algorithm 1) and dense sign.

Each pin compares the iterative oracle against dense linear algebra (LU
solves, eigendecomposition, Schur form), never against itself."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def tiny():
    dims = (2, 2, 3, 2)   # n = 288
    U = si.random_su3_links(dims, 0.7, 77)
    mu = 0.3
    A = O.dense_hw(dims, U, mu)
    b = si.gaussian_field(dims, 78)
    return dims, U, mu, A, b


def test_single_shift_is_a_linear_solve(tiny):
    """s = 1, no deflation: x = omega (A^2 - sigma)^{-1} A b, eqs. (2.2)-(2.3)."""
    dims, U, mu, A, b = tiny
    sigma, omega = np.array([-0.37]), np.array([1.7])
    x, rep, xs = O.fom_lr(dims, U, b, mu, sigma, omega, k=12, tol=1e-13, max_cycles=2000,
                          want_shifts=True)
    assert rep["converged"] and rep["cycles"] > 3        # restarts really happen
    ref = np.linalg.solve(A @ A - sigma[0] * np.eye(A.shape[0]), A @ b)
    assert _rel(xs[0], ref) < 1e-10
    assert _rel(x, omega[0] * ref) < 1e-10


def test_full_krylov_space_is_exact_in_one_cycle(tiny):
    """k >= n: the Arnoldi process spans the whole space and FOM is exact."""
    dims, U, mu, A, b = tiny
    n = A.shape[0]
    sigma, omega = O.kenney_laub(6, 0.5)
    x, rep, _ = O.fom_lr(dims, U, b, mu, sigma, omega, k=n + 4, tol=1e-12, max_cycles=1)
    assert rep["cycles"] == 1 and rep["breakdown"]
    ref = O.deflated_target(A, b, sigma, omega)
    assert _rel(x, ref) < 1e-9


def test_multishift_restarted_matches_dense(tiny):
    """Many shifts, many restarts, eq. (3.1)-(3.2): equals the dense rational target."""
    dims, U, mu, A, b = tiny
    sigma, omega = O.kenney_laub(16, 0.45)
    x, rep, xs = O.fom_lr(dims, U, b, mu, sigma, omega, k=10, tol=1e-13, max_cycles=5000,
                          want_shifts=True)
    assert rep["converged"] and rep["cycles"] > 5
    ref = O.deflated_target(A, b, sigma, omega)
    assert _rel(x, ref) < 1e-10
    # collinear residuals, eq. (3.1): stop after 3 cycles (far from converged)
    # and check that b~ - (A^2 - sigma_i) x_i all point along one vector
    _, rep3, xs3 = O.fom_lr(dims, U, b, mu, sigma, omega, k=10, tol=1e-13, max_cycles=3,
                            want_shifts=True)
    assert not rep3["converged"]
    bt = A @ b
    res = np.array([bt - (A @ (A @ xs3[i]) - sigma[i] * xs3[i]) for i in range(len(sigma))])
    big = res[np.argmax(np.linalg.norm(res, axis=1))]
    u = big / np.linalg.norm(big)
    assert np.linalg.norm(big) > 1e-6 * np.linalg.norm(bt)
    for r in res:
        perp = r - np.vdot(u, r) * u
        assert np.linalg.norm(perp) < 1e-12 * np.linalg.norm(bt)


def test_deflated_fomlr_matches_dense_target(lattice4):
    """FOM-LR(8,30) at 4^4, s = 16: equals the dense deflated target x*."""
    d = lattice4
    A, R, L, lam = d["A"], d["R"], d["L"], d["lam"]
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    x, rep, _ = O.fom_lr(d["dims"], d["U"], d["b"], d["mu"], sigma, omega, k=30, tol=1e-12,
                         R=R, L=L, lam=lam)
    assert rep["converged"]
    xstar = O.deflated_target(A, d["b"], sigma, omega, R, L, lam)
    assert _rel(x, xstar) < 1e-10
    # the Krylov part lives in range(I - P), eq. (4.5)
    c0 = L.conj().T @ d["b"]
    xP = R @ (np.sign(lam.real) * c0)
    assert np.linalg.norm(L.conj().T @ (x - xP)) < 1e-9 * np.linalg.norm(x)


def test_projection_toggle_runs(lattice4):
    """The variant without the projection step (Fig. 2) stays well defined."""
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    x1, r1, _ = O.fom_lr(d["dims"], d["U"], d["b"], d["mu"], sigma, omega, k=30, tol=1e-10,
                         R=d["R"], L=d["L"], lam=d["lam"], project_each_cycle=True)
    x0, r0, _ = O.fom_lr(d["dims"], d["U"], d["b"], d["mu"], sigma, omega, k=30, tol=1e-10,
                         max_cycles=r1["cycles"], R=d["R"], L=d["L"], lam=d["lam"],
                         project_each_cycle=False)
    assert r1["converged"] and np.all(np.isfinite(x0))


def test_dense_target_approximates_sign(lattice4):
    """x* agrees with exact sign(A) b within the rational error of Sec. 6.

    Bound: ||x* - sign(A) b|| <= kappa(X_rest) max |sign - g_s| ||(I-P) b||."""
    d = lattice4
    A = d["A"]
    a = abs(d["lam_next"][0])
    c = O.scale_from_bounds(a, 6.0)
    sigma, omega = O.kenney_laub(16, c)
    xstar = O.deflated_target(A, d["b"], sigma, omega, d["R"], d["L"], d["lam"])
    w, X, Xinv = d["eig"]
    exact = O.sign_eig(A, d["eig"]) @ d["b"]
    order = np.argsort(np.abs(w))
    keep = order[8:]
    kappa = np.linalg.cond(X[:, keep])
    err_fn = O.rational_error_bound(w[keep], 16, c)
    bound = kappa * err_fn * np.linalg.norm(d["b"])
    err = np.linalg.norm(xstar - exact)
    assert err <= bound * 1.01 + 1e-12
    assert err_fn < 1e-6
    # the deflated eigenvalues are the critical ones: the approximation is worst there
    assert O.rational_error_bound(w[order[:8]], 16, c) > err_fn


def test_dense_sign_invariants(lattice4):
    """sign(A)^2 = I and [sign(A), A] = 0 for the spectral sign at 4^4."""
    A = lattice4["A"]
    S = O.sign_eig(A, lattice4["eig"])
    n = A.shape[0]
    assert np.abs(S @ S - np.eye(n)).max() < 1e-9
    assert np.abs(S @ A - A @ S).max() < 1e-9


def test_schur_sign_equals_eigen_sign(tiny):
    """Two independent routes to sign(A): sorted Schur + Sylvester, and eigenvectors."""
    A = tiny[3]
    S1 = O.sign_eig(A)
    S2 = O.sign_schur(A)
    assert np.abs(S1 - S2).max() < 1e-10
    assert np.abs(S2 @ S2 - np.eye(A.shape[0])).max() < 1e-10


def test_critical_pairs(lattice4):
    d = lattice4
    A, R, L, lam = d["A"], d["R"], d["L"], d["lam"]
    assert np.abs(A @ R - R * lam).max() < 1e-12
    assert np.abs(L.conj().T @ A - lam[:, None] * L.conj().T).max() < 1e-10
    assert np.abs(L.conj().T @ R - np.eye(len(lam))).max() < 1e-10
    assert np.all(np.abs(lam) <= abs(d["lam_next"][0]) + 1e-15)


def _gm_setup(dims=(2, 2, 2, 2), mu=0.3, seed=61):
    U = si.random_su3_links(dims, 0.6, seed)
    A = O.dense_hw(dims, U, mu)
    b = si.gaussian_field(dims, seed + 1)
    return A, b


def test_gmres_lr_single_shift_is_minimal_residual():
    """s = 1, one cycle: the iterate minimises ||b~ - (A^2 - sigma) x|| over K_k(A^2, b~) (the
    defining property of GMRES), checked by least squares on an explicit power basis."""
    A, b = _gm_setup()
    n = A.shape[0]
    A2 = A @ A
    bt = A @ b
    sg, k = -0.7, 6
    x, cyc, _ = O.gmres_lr(A, b, [sg], [1.0], k, tol=1e-30, max_cycles=1)
    K = np.empty((n, k), dtype=np.complex128)
    v = bt / np.linalg.norm(bt)
    for j in range(k):
        K[:, j] = v
        v = A2 @ v
        v /= np.linalg.norm(v)
    M = (A2 - sg * np.eye(n)) @ K
    y = np.linalg.lstsq(M, bt, rcond=None)[0]
    assert cyc == 1
    assert np.linalg.norm(x - K @ y) < 1e-8 * np.linalg.norm(K @ y)


def test_gmres_lr_residuals_collinear_and_converges_to_target():
    """Multishift: after one cycle every shift's true residual is a multiple of the seed's
    (the collinearity that lets all shifts share one Krylov space); run to convergence, the
    deflated sum equals the dense target of eqs. (4.2)-(4.3) with (6.2)."""
    A, b = _gm_setup()
    n = A.shape[0]
    A2 = A @ A
    bt = A @ b
    sigma, omega = O.kenney_laub(5, 1.0)
    k = 8
    # per-shift iterates from one cycle: weights e_i pick one shift at a time
    res = []
    for i in range(len(sigma)):
        w = np.zeros(len(sigma))
        w[i] = 1.0
        xi, _, _ = O.gmres_lr(A, b, sigma, w, k, tol=1e-30, max_cycles=1)
        res.append(bt - (A2 - sigma[i] * np.eye(n)) @ xi)
    seed = int(np.argmin(np.abs(sigma)))
    r0 = res[seed]
    for i, ri in enumerate(res):
        coef = np.vdot(r0, ri) / np.vdot(r0, r0)
        assert np.linalg.norm(ri - coef * r0) < 1e-9 * np.linalg.norm(ri)
    R, L, lam, _ = O.critical_eigenpairs(A, 6, extra=1)
    x, cyc, rr = O.gmres_lr(A, b, sigma, omega, k, tol=1e-11, max_cycles=500, R=R, L=L, lam=lam)
    xt = O.deflated_target(A, b, sigma, omega, R, L, lam)
    assert cyc > 1 and np.max(rr) <= 1e-11
    assert np.linalg.norm(x - xt) < 1e-9 * np.linalg.norm(xt)
