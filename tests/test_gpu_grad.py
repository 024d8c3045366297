"""Gradients of Re<c, sign(H_W(mu)) b> (SignApply): b-gradient by the adjoint solve,
mu-gradient by per-shift forward and adjoint iterates (undeflated function).

Checked against the oracle's dense Daleckii-Krein derivative on a small lattice
and central finite differences of the oracle with step 1e-4 at 6^4 (mu = 0.5)."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(dims, U, mu, sigma, omega, k=20, tol=1e-13):
    import paper_0910_2927_gb300 as pkg
    ctx = pkg.SignContext(dims, mu=mu)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_rational(sigma, omega)
    ctx.set_restart(k=k, tol=tol, max_cycles=5000)
    return ctx


def test_dhw_dmu_matches_central_difference():
    from paper_0910_2927_gb300.autograd import dhw_dmu
    dims, mu, h = (3, 2, 3, 4), 0.4, 1e-5
    U = si.random_su3_links(dims, 0.7, 51)
    v = si.gaussian_field(dims, 52)
    fd = (O.hw(dims, U, v, mu + h) - O.hw(dims, U, v, mu - h)) / (2 * h)
    sigma, omega = O.kenney_laub(4, 0.5)
    with _ctx(dims, U, mu, sigma, omega) as ctx:
        got = dhw_dmu(ctx, torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.linalg.norm(got - fd) < 1e-8 * np.linalg.norm(fd)


def test_gradients_match_dense_daleckii_krein():
    """Dense reference (oracle deflated_sign_derivative with m = 0): A = X diag(l) X^{-1},
    F(A) = X f(l) X^{-1} with f(t) = t sum omega/(t^2 - sigma); dF[E] = X (F^ o (X^{-1} E X)) X^{-1},
    F^_jk = divided differences of f, along E = A' (oracle dense_dhw_dmu)."""
    from paper_0910_2927_gb300.autograd import SignApply
    dims, mu = (3, 2, 3, 4), 0.5
    U = si.random_su3_links(dims, 0.7, 53)
    b = si.gaussian_field(dims, 54)
    c = si.gaussian_field(dims, 55)
    sigma, omega = O.kenney_laub(12, 0.4)
    A = O.dense_hw(dims, U, mu)
    F, dF = O.deflated_sign_derivative(A, O.dense_dhw_dmu(dims, U, mu), sigma, omega, m=0)
    dmu_ref = np.real(np.vdot(c, dF @ b))
    gb_ref = F.conj().T @ c
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    with _ctx(dims, U, mu, sigma, omega) as ctx:
        x = SignApply.apply(bt, mut, ctx)
        loss = torch.vdot(torch.from_numpy(c).cuda(), x).real
        loss.backward()
    gb = bt.grad.cpu().numpy()
    assert np.linalg.norm(gb - gb_ref) < 1e-9 * np.linalg.norm(gb_ref)
    assert abs(float(mut.grad) - dmu_ref) < 1e-7 * max(1.0, abs(dmu_ref))


def test_config4_finite_differences():
    """6^4, mu = 0.5: d/dmu Re<c, x> against central differences of the oracle, h = 1e-4."""
    from paper_0910_2927_gb300.autograd import SignApply
    dims, mu, h = (6, 6, 6, 6), 0.5, 1e-4
    g_seed, b_seed, c_seed = si.CONFIG_SEEDS[4]
    U = si.random_su3_links(dims, 0.7, g_seed)
    b = si.gaussian_field(dims, b_seed)
    c = si.gaussian_field(dims, c_seed)
    sigma, omega = O.kenney_laub(20, 0.3)
    def loss_oracle(m):
        x, rep, _ = O.fom_lr(dims, U, b, m, sigma, omega, k=40, tol=1e-12, max_cycles=3000)
        assert rep["converged"]
        return np.real(np.vdot(c, x))
    fd = (loss_oracle(mu + h) - loss_oracle(mu - h)) / (2 * h)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    with _ctx(dims, U, mu, sigma, omega, k=40, tol=1e-12) as ctx:
        x = SignApply.apply(bt, mut, ctx)
        loss = torch.vdot(torch.from_numpy(c).cuda(), x).real
        loss.backward()
        # b-gradient: directional derivative along a random direction against the oracle
        d = si.gaussian_field(dims, 99)
    xo_p, _, _ = O.fom_lr(dims, U, b + 1e-3 * d, mu, sigma, omega, k=40, tol=1e-12, max_cycles=3000)
    xo_m, _, _ = O.fom_lr(dims, U, b - 1e-3 * d, mu, sigma, omega, k=40, tol=1e-12, max_cycles=3000)
    dir_fd = np.real(np.vdot(c, xo_p - xo_m)) / 2e-3
    dir_ad = np.real(np.vdot(bt.grad.cpu().numpy(), d))
    assert abs(float(mut.grad) - fd) < 1e-5 * max(1.0, abs(fd))
    assert abs(dir_ad - dir_fd) < 1e-5 * max(1.0, abs(dir_fd))


@pytest.mark.parametrize("mu,m", [(0.5, 6), (0.3, 10)])
def test_deflated_gradient_matches_dense_daleckii_krein(mu, m):
    """With m deflated pairs (and 4 extra ones set for the derivative) the forward applies
    F = X f~(Lambda) X^{-1}, f~ = sign(Re lambda)
    on the deflated eigenvalues and g elsewhere (g(t) = t sum omega / (t^2 - sigma)).  Its
    derivative along A' is X (F^ o (X^{-1} A' X)) X^{-1} with the divided differences of f~:
    the motion of the deflated eigenvectors is in the off-diagonal terms between deflated and
    undeflated eigenvalues.  The GPU gradient (forward and adjoint solves, complex-shift
    solves for the reduced resolvents) must match it."""
    from paper_0910_2927_gb300.autograd import SignApply
    dims = (3, 2, 3, 4)
    U = si.random_su3_links(dims, 0.7, 57)
    b = si.gaussian_field(dims, 58)
    c = si.gaussian_field(dims, 59)
    sigma, omega = O.kenney_laub(12, 0.4)
    A = O.dense_hw(dims, U, mu)
    dec = O.eig(A)
    e = 4  # the next eigenpairs, kept for the reduced resolvents of the derivative
    Ra, La, lama, _ = O.critical_eigenpairs(A, m + e, decomposition=dec)
    R, L, lam = Ra[:, :m], La[:, :m], lama[:m]
    F, dF = O.deflated_sign_derivative(A, O.dense_dhw_dmu(dims, U, mu), sigma, omega, m=m, decomposition=dec)
    dmu_ref = np.real(np.vdot(c, dF @ b))
    x_ref = F @ b
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    with _ctx(dims, U, mu, sigma, omega) as ctx:
        ctx.set_deflation(R, L, lam, extra=(Ra[:, m:], La[:, m:], lama[m:]))
        x = SignApply.apply(bt, mut, ctx)
        assert np.linalg.norm(x.detach().cpu().numpy() - x_ref) < 1e-9 * np.linalg.norm(x_ref)
        loss = torch.vdot(torch.from_numpy(c).cuda(), x).real
        loss.backward()
    gb_ref = F.conj().T @ c
    assert np.linalg.norm(bt.grad.cpu().numpy() - gb_ref) < 1e-9 * np.linalg.norm(gb_ref)
    assert abs(float(mut.grad) - dmu_ref) < 1e-7 * max(1.0, abs(dmu_ref)), (float(mut.grad), dmu_ref)


def test_config4_deflated_finite_differences():
    """6^4, mu = 0.5, m = 20 deflated pairs (4 extra for the reduced resolvents), from the GPU
    eigensolver at mu and at mu +- h (the context rebuilds them when SignApply or set_mu moves mu).
    The oracle's central difference, h = 1e-4, of Re<c, x(mu)> with x from its own FOM-LR on the
    rebuilt pairs (each pair checked against the oracle's stencil), against the GPU's mu-gradient,
    whose eigenvector-motion terms are what the deflation adds (Sec. 4, eqs. 4.2-4.3)."""
    import math
    from paper_0910_2927_gb300.autograd import SignApply
    import paper_0910_2927_gb300 as pkg
    dims, mu, h, m = (6, 6, 6, 6), 0.5, 1e-4, 20
    g_seed, b_seed, c_seed = si.CONFIG_SEEDS[4]
    U = si.random_su3_links(dims, 0.7, g_seed)
    b = si.gaussian_field(dims, b_seed)
    c = si.gaussian_field(dims, c_seed)
    with _ctx(dims, U, mu, *O.kenney_laub(1, 1.0), k=40, tol=1e-12) as ctx:
        # set-up accuracy: the deflated function moves by ~1e-2 x the eigen-residual (measured on
        # 4^4), so 1e-10 keeps the difference quotient's error near 1e-10 / (2h) * 1e-2 = 5e-9
        lam = ctx.build_deflation(m, extra=4, eig_tol=1e-10)
        b_max = abs(4.0 - 1.6) + 3.0 * math.sqrt(2.0) + math.sqrt(2.0 * math.cosh(2.0 * mu))
        sigma, omega = pkg.kenney_laub(20, 1.0 / math.sqrt(abs(lam[m]) * b_max))
        ctx.set_rational(sigma, omega)
        bt = torch.from_numpy(b).cuda().requires_grad_(True)
        mut = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
        x = SignApply.apply(bt, mut, ctx)
        loss = torch.vdot(torch.from_numpy(c).cuda(), x).real
        loss.backward()
        pairs = {}
        for mm in (mu + h, mu - h):
            ctx.set_mu(mm, rebuild_deflation=True)
            pairs[mm] = ctx.get_deflation()
        assert ctx.m == m
    def loss_oracle(mm):
        R, L, lm = pairs[mm]
        for j in (0, m - 1):
            rr = O.hw(dims, U, R[:, j], mm) - lm[j] * R[:, j]
            assert np.linalg.norm(rr) <= 1e-9 * abs(lm[j]) * np.linalg.norm(R[:, j])
        xo, rep, _ = O.fom_lr(dims, U, b, mm, sigma, omega, k=40, tol=1e-13, max_cycles=3000, R=R, L=L, lam=lm)
        assert rep["converged"]
        return np.real(np.vdot(c, xo))
    fd = (loss_oracle(mu + h) - loss_oracle(mu - h)) / (2 * h)
    assert abs(float(mut.grad) - fd) < 1e-5 * max(1.0, abs(fd)), (float(mut.grad), fd)
