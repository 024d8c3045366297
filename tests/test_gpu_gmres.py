"""GPU parity of GMRES-LR (restarted multishift GMRES with LR deflation, Sec. 2 and Sec. 4):
the seed shift (smallest |sigma|) by minimal residual, the others by the bordered systems that
keep their residuals collinear.  Against the oracle's gmres_lr on the same seeded inputs: the
per-shift iterates after a fixed number of cycles (the caller's shift order restored), the
converged deflated solve, and the dense target."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_FP64 = 1e-10


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def small():
    dims, mu = (3, 2, 3, 4), 0.3   # n = 864: several CTA tiles and a ragged tail
    U = si.random_su3_links(dims, 0.7, 21)
    A = O.dense_hw(dims, U, mu)
    R, L, lam, nxt = O.critical_eigenpairs(A, 6, extra=2)
    return dict(dims=dims, mu=mu, U=U, A=A, R=R, L=L, lam=lam, nxt=nxt)


def _ctx(d, sigma, omega, k, tol, max_cycles):
    import paper_0910_2927_gb300 as pkg
    ctx = pkg.SignContext(d["dims"], mu=d["mu"])
    ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
    ctx.set_rational(sigma, omega)
    ctx.set_restart(k=k, tol=tol, max_cycles=max_cycles)
    ctx.set_method(pkg.METHOD_GMRES)
    return ctx


def test_shift_iterates_after_fixed_cycles(small):
    d = small
    sigma, omega = O.kenney_laub(8, 0.5)
    sigma = sigma[::-1].copy()     # the seed (smallest |sigma|) is not the first shift
    omega = omega[::-1].copy()
    b = si.gaussian_field(d["dims"], 24)
    with _ctx(d, sigma, omega, k=8, tol=1e-14, max_cycles=3) as ctx:
        x, xs, rep = ctx.apply(torch.from_numpy(b).cuda(), shifts=True)
        xs = xs.cpu().numpy()[:, 0]
        x = x.cpu().numpy()[0] if x.dim() == 2 else x.cpu().numpy()
    xo, cyc, _, Xo = O.gmres_lr(d["A"], b, sigma, omega, 8, tol=1e-14, max_cycles=3, want_shifts=True)
    assert rep["status"] == 3 and rep["cycles"] == 3 == cyc
    for i in range(len(sigma)):
        assert _rel(xs[i], Xo[i]) < TOL_FP64
    assert _rel(x, xo) < TOL_FP64


@pytest.mark.parametrize("adjoint", [False, True])
def test_deflated_converged(small, adjoint):
    d = small
    c = O.scale_from_bounds(abs(d["nxt"][0]), 6.5)
    sigma, omega = O.kenney_laub(16, c)
    b = si.gaussian_field(d["dims"], 23)
    with _ctx(d, sigma, omega, k=12, tol=1e-12, max_cycles=2000) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        x, rep = ctx.apply(torch.from_numpy(b).cuda(), adjoint=adjoint)
        x = x.cpu().numpy()
    if adjoint:
        Aop, R, L, lam = d["A"].conj().T, d["L"], d["R"], np.conj(d["lam"])
    else:
        Aop, R, L, lam = d["A"], d["R"], d["L"], d["lam"]
    xo, cyc, rr = O.gmres_lr(Aop, b, sigma, omega, 12, tol=1e-12, max_cycles=2000, R=R, L=L, lam=lam)
    assert rep["status"] == 0 and rep["cycles"] == cyc
    assert _rel(x, xo) < TOL_FP64
    assert _rel(x, O.deflated_target(Aop, b, sigma, omega, R, L, lam)) < 1e-9


def test_gmres_refuses_mixed_and_split(small):
    import paper_0910_2927_gb300 as pkg
    d = small
    sigma, omega = O.kenney_laub(6, 0.5)
    b = torch.from_numpy(si.gaussian_field(d["dims"], 25)).cuda()
    with _ctx(d, sigma, omega, k=8, tol=1e-10, max_cycles=100) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8)
        with pytest.raises(pkg.SignError):
            ctx.apply(b)
        ctx.set_precision(pkg.PREC_FP64)
        ctx.set_formulation(pkg.FORM_A)
        with pytest.raises(pkg.SignError):
            ctx.apply(b)
        ctx.set_formulation(pkg.FORM_A2)
        x, rep = ctx.apply(b)
        assert rep["status"] == 0
        with pytest.raises(pkg.SignError):
            ctx.set_method(7)


def test_single_shift_and_deflated_subspace(small):
    """s = 1 (no bordered systems: plain restarted GMRES on one shifted system) against the
    oracle; a right-hand side inside the deflated subspace gives x = x_P exactly."""
    d = small
    sigma, omega = np.array([-0.35]), np.array([0.8])
    b = si.gaussian_field(d["dims"], 26)
    with _ctx(d, sigma, omega, k=10, tol=1e-12, max_cycles=2000) as ctx:
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        bP = d["R"] @ np.arange(1, 7)
        xp, repp = ctx.apply(torch.from_numpy(bP).cuda())
    xo, cyc, _ = O.gmres_lr(d["A"], b, sigma, omega, 10, tol=1e-12, max_cycles=2000)
    assert rep["status"] == 0 and rep["cycles"] == cyc
    assert _rel(x.cpu().numpy(), xo) < TOL_FP64
    xP = d["R"] @ (np.sign(d["lam"].real) * np.arange(1, 7))
    assert _rel(xp.cpu().numpy(), xP) < 1e-10
