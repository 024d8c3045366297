"""Pins for the oracle's Wilson kernel H_W(mu) = gamma5 D_W(mu) (Sec. 1).

Checked against things other than itself: the free-field plane-wave closed
form (fixes every sign, the e^{+-mu} placement and the boundary phase), the
identity H_W(mu)^dag = H_W(-mu), Hermiticity at mu = 0, and gauge covariance
(fixes U versus U^dag on forward and backward hops)."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

# gamma matrices written out from the chiral-basis definition
_S = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
_G = []
for k in range(3):
    g = np.zeros((4, 4), dtype=complex)
    g[:2, 2:] = -1j * _S[k]
    g[2:, :2] = 1j * _S[k]
    _G.append(g)
_gt = np.zeros((4, 4), dtype=complex)
_gt[:2, 2:] = np.eye(2)
_gt[2:, :2] = np.eye(2)
_G.append(_gt)
_G5 = _G[0] @ _G[1] @ _G[2] @ _G[3]


def test_gamma_algebra():
    for a in range(4):
        for b in range(4):
            ac = _G[a] @ _G[b] + _G[b] @ _G[a]
            np.testing.assert_allclose(ac, 2 * np.eye(4) * (a == b), atol=1e-15)
        np.testing.assert_allclose(_G[a], _G[a].conj().T, atol=0)
    np.testing.assert_allclose(_G5, np.diag([1, 1, -1, -1]), atol=1e-15)


def _coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(range(lt), range(lz), range(ly), range(lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0])
@pytest.mark.parametrize("dims,ap", [((4, 4, 4, 4), (0, 0, 0, 1)), ((3, 4, 5, 6), (0, 0, 0, 1)),
                                     ((4, 3, 2, 5), (1, 0, 1, 0))])
def test_free_field_plane_wave(mu, dims, ap):
    """U = 1: H_W psi = gamma5 [(4+m) - sum cos q + i sum gamma sin q] psi, q_t = p_t - i mu."""
    mass = -1.6
    U = si.unit_links(dims)
    X = _coords(dims)
    rng = np.random.default_rng(5)
    for trial in range(4):
        nvec = [rng.integers(0, d) for d in dims]
        p = np.array([(2 * np.pi * nvec[i] + (np.pi if ap[i] else 0.0)) / dims[i] for i in range(4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * X @ p)
        psi = (phase[:, None, None] * u[None]).reshape(-1)
        q = p.astype(complex)
        q[3] = p[3] - 1j * mu
        Dp = (4 + mass - np.sum(np.cos(q))) * np.eye(4) + 1j * sum(_G[i] * np.sin(q[i]) for i in range(4))
        expect = (phase[:, None, None] * (_G5 @ Dp @ u)[None]).reshape(-1)
        got = O.hw(dims, U, psi, mu, mass, ap)
        np.testing.assert_allclose(got, expect, atol=1e-12 * np.abs(expect).max())


def test_gamma5_hermiticity_and_mu0_hermiticity():
    dims = (3, 4, 3, 4)
    U = si.random_su3_links(dims, 0.7, 42)
    b = si.gaussian_field(dims, 1)
    c = si.gaussian_field(dims, 2)
    for mu in (0.3, 1.0):
        lhs = np.vdot(c, O.hw(dims, U, b, mu))
        rhs = np.vdot(O.hw(dims, U, c, -mu), b)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
        # and not Hermitian at mu != 0
        assert abs(lhs - np.vdot(O.hw(dims, U, c, mu), b)) > 1e-3 * abs(lhs)
    lhs = np.vdot(c, O.hw(dims, U, b, 0.0))
    rhs = np.vdot(O.hw(dims, U, c, 0.0), b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gauge_covariance():
    """U^G_nu(x) = G(x) U_nu(x) G(x+nu)^dag  =>  H[U^G] (G psi) = G H[U] psi."""
    dims = (4, 3, 4, 5)
    U = si.random_su3_links(dims, 0.7, 9)
    G = si.random_gauge_transform(dims, 10)
    X = _coords(dims)
    vol = X.shape[0]
    strides = np.array([1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]])
    UG = np.empty_like(U)
    for nu in range(4):
        Y = X.copy()
        Y[:, nu] = (Y[:, nu] + 1) % dims[nu]
        fwd = Y @ strides
        UG[:, nu] = G @ U[:, nu] @ np.conj(np.transpose(G[fwd], (0, 2, 1)))
    psi = si.gaussian_field(dims, 3).reshape(vol, 4, 3)
    Gpsi = np.einsum("sab,sxb->sxa", G, psi).reshape(-1)
    for mu in (0.0, 0.4):
        lhs = O.hw(dims, UG, Gpsi, mu)
        rhs = np.einsum("sab,sxb->sxa", G, O.hw(dims, U, psi.reshape(-1), mu).reshape(vol, 4, 3)).reshape(-1)
        np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())


def test_sites_subset_matches_full():
    dims = (3, 4, 5, 2)
    U = si.random_su3_links(dims, 0.7, 4)
    psi = si.gaussian_field(dims, 5)
    full = O.hw(dims, U, psi, 0.3).reshape(-1, 12)
    sites = np.array([0, 7, 33, 119])
    np.testing.assert_array_equal(O.hw_sites(dims, U, psi, sites, 0.3), full[sites])


def test_overlap_ginsparg_wilson_and_circle():
    """D_ov = 1 + gamma5 sign(H_W) with the exact sign satisfies the Ginsparg-Wilson relation
    gamma5 D + D gamma5 = D gamma5 D at any mu (it needs only sign^2 = 1); at mu = 0 (H_W
    Hermitian) D_ov is normal with its spectrum on the circle |z - 1| = 1.  A wrong gamma5
    (another spin order or sign) breaks both."""
    dims = (2, 2, 2, 2)
    vol = 16
    U = si.random_su3_links(dims, 0.6, 71)
    g5 = np.diag(O.gamma5_diag(vol))
    for mu in (0.0, 0.35):
        A = O.dense_hw(dims, U, mu)
        D = O.overlap_dense(O.sign_eig(A), vol)
        lhs = g5 @ D + D @ g5
        assert np.linalg.norm(lhs - D @ g5 @ D) < 1e-10 * np.linalg.norm(lhs)
        if mu == 0.0:
            assert np.linalg.norm(D @ D.conj().T - D.conj().T @ D) < 1e-10 * np.linalg.norm(D) ** 2
            z = np.linalg.eigvals(D)
            assert np.max(np.abs(np.abs(z - 1.0) - 1.0)) < 1e-10
    # gamma5 H_W is D_W: its hermiticity at mu = 0 fixes the gamma5 of H_W = gamma5 D_W
    A0 = O.dense_hw(dims, U, 0.0)
    assert np.linalg.norm(A0 - A0.conj().T) < 1e-12 * np.linalg.norm(A0)
    Dw = g5 @ A0
    assert np.linalg.norm(g5 @ Dw @ g5 - Dw.conj().T) < 1e-12 * np.linalg.norm(Dw)


def test_deflated_sign_matrix_matches_deflated_target():
    """The dense F(A) applied to b equals the deflated target built by shifted LU solves."""
    dims, mu = (2, 2, 2, 2), 0.3
    U = si.random_su3_links(dims, 0.6, 72)
    A = O.dense_hw(dims, U, mu)
    b = si.gaussian_field(dims, 73)
    sigma, omega = O.kenney_laub(8, 0.5)
    dec = O.eig(A)
    R, L, lam, _ = O.critical_eigenpairs(A, 5, decomposition=dec)
    F = O.deflated_sign_matrix(A, sigma, omega, m=5, decomposition=dec)
    xt = O.deflated_target(A, b, sigma, omega, R, L, lam)
    assert np.linalg.norm(F @ b - xt) < 1e-10 * np.linalg.norm(xt)
    F0 = O.deflated_sign_matrix(A, sigma, omega, m=0, decomposition=dec)
    xt0 = O.deflated_target(A, b, sigma, omega)
    assert np.linalg.norm(F0 @ b - xt0) < 1e-10 * np.linalg.norm(xt0)


def test_dense_dhw_dmu_against_richardson_difference():
    """A' from the exact sinh form against a fourth-order central difference of the C stencil
    (no shared arithmetic: the stencil is the oracle's C code, the dense matrix its NumPy build)."""
    dims, mu = (2, 2, 3, 2), 0.45
    U = si.random_su3_links(dims, 0.6, 74)
    v = si.gaussian_field(dims, 75)
    Ad = O.dense_dhw_dmu(dims, U, mu)
    h = 1e-2
    d1 = (O.hw(dims, U, v, mu + h) - O.hw(dims, U, v, mu - h)) / (2 * h)
    d2 = (O.hw(dims, U, v, mu + 2 * h) - O.hw(dims, U, v, mu - 2 * h)) / (4 * h)
    rich = (4 * d1 - d2) / 3
    assert np.linalg.norm(Ad @ v - rich) < 1e-8 * np.linalg.norm(rich)
    # the sinh form is exact, so the step does not matter (a plain central difference would
    # change by O(h^2) between these steps)
    assert np.linalg.norm(O.dense_dhw_dmu(dims, U, mu) - O.dense_dhw_dmu(dims, U, mu, h=0.3)) \
        < 1e-12 * np.linalg.norm(Ad)


def test_frechet_closed_forms():
    """Daleckii-Krein with f(t) = t^2 gives A E + E A, with f(t) = t^3 gives A^2 E + A E A + E A^2."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    E = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    dec = O.eig(A)
    w = dec[0]
    d2 = O.frechet_dense(E, w ** 2, 2 * w, dec)
    assert np.linalg.norm(d2 - (A @ E + E @ A)) < 1e-10 * np.linalg.norm(A @ E)
    d3 = O.frechet_dense(E, w ** 3, 3 * w ** 2, dec)
    ref3 = A @ A @ E + A @ E @ A + E @ A @ A
    assert np.linalg.norm(d3 - ref3) < 1e-10 * np.linalg.norm(ref3)


def test_deflated_sign_derivative_against_mu_difference():
    """d/dmu of the dense deflated sign matrix (eigendecompositions recomputed at mu +- h, the m
    critical pairs re-selected) equals the Daleckii-Krein derivative along A', undeflated and
    deflated; F is the same matrix deflated_sign_matrix builds."""
    dims, mu = (2, 2, 2, 3), 0.4
    U = si.random_su3_links(dims, 0.6, 76)
    sigma, omega = O.kenney_laub(8, 0.5)
    A = O.dense_hw(dims, U, mu)
    Ad = O.dense_dhw_dmu(dims, U, mu)
    dec = O.eig(A)
    h = 1e-5
    for m in (0, 5):
        F, dF = O.deflated_sign_derivative(A, Ad, sigma, omega, m=m, decomposition=dec)
        assert np.linalg.norm(F - O.deflated_sign_matrix(A, sigma, omega, m=m, decomposition=dec)) \
            < 1e-13 * np.linalg.norm(F)
        Fp = O.deflated_sign_matrix(O.dense_hw(dims, U, mu + h), sigma, omega, m=m)
        Fm = O.deflated_sign_matrix(O.dense_hw(dims, U, mu - h), sigma, omega, m=m)
        fd = (Fp - Fm) / (2 * h)
        assert np.linalg.norm(dF - fd) < 1e-6 * np.linalg.norm(fd)
