"""Pins for the oracle's rational approximation (Sec. 6, eqs. (6.1)-(6.2)).

The partial fractions of eq. (6.2) are checked against the closed form of
eq. (6.1), which is an independent expression of the same function."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si


@pytest.mark.parametrize("s", [1, 2, 7, 16, 20])
def test_partial_fractions_equal_closed_form(s):
    rng = np.random.default_rng(s)
    t = rng.standard_normal(200) * 2 + 1j * rng.standard_normal(200)
    t = t[np.abs(t.real) > 0.05]
    g_pf = O.kl_partial_fractions(t, s)
    g_cf = O.kl_closed_form(t, s)
    np.testing.assert_allclose(g_pf, g_cf, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("c", [0.3, 1.0, 2.5])
def test_scale_folding(c):
    """g_s(c t) from the folded (sigma', omega') equals eq. (6.1) at c t."""
    s = 16
    rng = np.random.default_rng(7)
    t = rng.standard_normal(100) + 0.3j * rng.standard_normal(100)
    np.testing.assert_allclose(O.kl_partial_fractions(t, s, c), O.kl_closed_form(c * t, s),
                               rtol=1e-12, atol=1e-13)


def test_coefficients_closed_form_values():
    """s = 1: theta = pi/4, omega = 2, sigma = -1, so g_1(t) = 2t/(t^2+1)."""
    sig, om = O.kenney_laub(1, 1.0)
    assert sig[0] == pytest.approx(-1.0, abs=1e-15)
    assert om[0] == pytest.approx(2.0, abs=1e-15)
    sig, om = O.kenney_laub(2, 1.0)   # theta = pi/8, 3pi/8
    t1, t2 = np.tan(np.pi / 8), np.tan(3 * np.pi / 8)
    np.testing.assert_allclose(sig, [-t1 ** 2, -t2 ** 2], rtol=1e-14)
    np.testing.assert_allclose(om, [0.5 / np.cos(np.pi / 8) ** 2, 0.5 / np.cos(3 * np.pi / 8) ** 2],
                               rtol=1e-14)
    # shifts negative real and increasing in magnitude
    sig, om = O.kenney_laub(20, 1.0)
    assert np.all(sig < 0) and np.all(np.diff(sig) < 0) and np.all(om > 0)


@pytest.mark.parametrize("s", [4, 16])
def test_sign_limits(s):
    """g_s(1) = 1 exactly, g_s is odd, and g_s(t) -> sign(Re t) as s grows."""
    assert O.kl_partial_fractions(np.array([1.0]), s)[0] == pytest.approx(1.0, abs=1e-14)
    rng = np.random.default_rng(3)
    t = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    np.testing.assert_allclose(O.kl_partial_fractions(-t, s), -O.kl_partial_fractions(t, s),
                               rtol=1e-13)
    t = np.array([0.5, 2.0, -1.5 + 0.2j, 0.8 - 0.3j])
    g = O.kl_partial_fractions(t, 64)
    np.testing.assert_allclose(g, np.sign(t.real), atol=1e-10)


def test_error_bound_matches_direct_evaluation():
    """|sign - g_s| from the closed form q-expression equals direct evaluation."""
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(300) * 3 + 0.5j * rng.standard_normal(300)
    lam = lam[np.abs(lam.real) > 0.2]
    for s, c in [(16, 0.6), (20, 0.3)]:
        direct = np.max(np.abs(np.sign(lam.real) - O.kl_closed_form(c * lam, s)))
        assert O.rational_error_bound(lam, s, c) == pytest.approx(direct, rel=1e-6, abs=1e-15)


def test_roberts_newton_sign_is_the_spectral_sign():
    """Roberts' iteration on a random non-normal matrix equals sign(M) = X sign(Re L) X^{-1}."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    S = O.roberts_newton_sign(M)
    w, X = np.linalg.eig(M)
    ref = (X * np.where(w.real > 0, 1.0, -1.0)) @ np.linalg.inv(X)
    assert np.linalg.norm(S - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(S @ S - np.eye(12)) < 1e-10 * 12


def test_direct_projection_exact_at_full_dimension():
    """Eq. (6.3) with k = n (the Krylov space is the whole space) gives sign(A) b; with
    deflation the deflated part is exact at any k and the error falls as k grows."""
    dims, mu = (2, 2, 2, 2), 0.4
    U = si.random_su3_links(dims, 0.6, 81)
    A = O.dense_hw(dims, U, mu)
    b = si.gaussian_field(dims, 82)
    xs = O.sign_eig(A) @ b
    n = A.shape[0]
    assert np.linalg.norm(O.direct_projection(A, b, n) - xs) < 1e-9 * np.linalg.norm(xs)
    R, L, lam, _ = O.critical_eigenpairs(A, 6, extra=1)
    errs = [np.linalg.norm(O.direct_projection(A, b, k, R, L, lam) - xs) for k in (16, 48, n)]
    assert errs[2] < 1e-9 * np.linalg.norm(xs) and errs[1] < errs[0]
