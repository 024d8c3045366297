"""GPU parity of sign(H_W(mu)) b by restarted FOM-LR (Algorithm 1), FP64 form.

The CUDA path and the oracle run the same algorithm on the same seeded inputs
with a tight stopping tolerance; their results agree to relative 2-norm
error <= 1e-10 (the FP64 bar)."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_FP64 = 1e-10


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ctx(dims, U, mu, sigma, omega, k, tol, max_cycles=2000, project=True):
    import paper_0910_2927_gb300 as pkg
    ctx = pkg.SignContext(dims, mu=mu)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_rational(sigma, omega)
    ctx.set_restart(k=k, tol=tol, max_cycles=max_cycles, project_each_cycle=project)
    return ctx


@pytest.fixture(scope="module")
def small():
    dims, mu = (3, 2, 3, 4), 0.3   # n = 864: several CTA tiles and a ragged tail
    U = si.random_su3_links(dims, 0.7, 21)
    A = O.dense_hw(dims, U, mu)
    dec = O.eig(A)
    R, L, lam, nxt = O.critical_eigenpairs(A, 6, extra=2, decomposition=dec)
    return dict(dims=dims, mu=mu, U=U, A=A, R=R, L=L, lam=lam, nxt=nxt)


def test_no_deflation_matches_oracle(small):
    d = small
    sigma, omega = O.kenney_laub(12, 0.4)
    b = si.gaussian_block(d["dims"], 2, 22)
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=10, tol=1e-12) as ctx:
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        x = x.cpu().numpy()
    assert rep["status"] == 0 and rep["cycles"] > 2
    for r in range(2):
        xo, orep, _ = O.fom_lr(d["dims"], d["U"], b[r], d["mu"], sigma, omega, k=10, tol=1e-12, max_cycles=2000)
        assert _rel(x[r], xo) < TOL_FP64
        assert _rel(x[r], O.deflated_target(d["A"], b[r], sigma, omega)) < 1e-9


@pytest.mark.parametrize("project", [True, False])
def test_deflated_matches_oracle(small, project):
    d = small
    c = O.scale_from_bounds(abs(d["nxt"][0]), 6.5)
    sigma, omega = O.kenney_laub(16, c)
    b = si.gaussian_field(d["dims"], 23)
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=12, tol=1e-12, project=project) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        x = x.cpu().numpy()
    xo, orep, _ = O.fom_lr(d["dims"], d["U"], b, d["mu"], sigma, omega, k=12, tol=1e-12, max_cycles=2000,
                           project_each_cycle=project, R=d["R"], L=d["L"], lam=d["lam"])
    assert rep["cycles"] == orep["cycles"]
    assert _rel(x, xo) < TOL_FP64
    if project:
        assert _rel(x, O.deflated_target(d["A"], b, sigma, omega, d["R"], d["L"], d["lam"])) < 1e-9


def test_config1_4x4x4x4(lattice4):
    """The 4^4 plain-FP64 workload: s = 16, k = 30, m = 8, mu = 0.3."""
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=30, tol=1e-12) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        x, rep = ctx.apply(torch.from_numpy(d["b"]).cuda())
        x = x.cpu().numpy()
        xh, reph = ctx.apply(d["b"])        # host buffers through the same ABI call
    xo, orep, _ = O.fom_lr(d["dims"], d["U"], d["b"], d["mu"], sigma, omega, k=30, tol=1e-12,
                           R=d["R"], L=d["L"], lam=d["lam"])
    assert _rel(x, xo) < TOL_FP64
    assert _rel(xh, xo) < TOL_FP64
    xstar = O.deflated_target(d["A"], d["b"], sigma, omega, d["R"], d["L"], d["lam"])
    assert _rel(x, xstar) < 1e-9


def test_shift_iterates_and_collinearity(small):
    d = small
    sigma, omega = O.kenney_laub(8, 0.5)
    b = si.gaussian_field(d["dims"], 24)
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=8, tol=1e-13, max_cycles=4) as ctx:
        x, xs, rep = ctx.apply(torch.from_numpy(b).cuda(), shifts=True)
        xs = xs.cpu().numpy()[:, 0]
    _, _, xso = O.fom_lr(d["dims"], d["U"], b, d["mu"], sigma, omega, k=8, tol=1e-13, max_cycles=4,
                         want_shifts=True)
    assert rep["status"] == 3   # stopped by max_cycles: NOT_CONVERGED, last iterate returned
    for i in range(len(sigma)):
        assert _rel(xs[i], xso[i]) < TOL_FP64


def test_adjoint_is_sign_at_minus_mu(small):
    """sign(A)^dag c via SGN_APPLY_ADJOINT equals the oracle run on H_W(-mu) with L, R swapped."""
    d = small
    c = O.scale_from_bounds(abs(d["nxt"][0]), 6.5)
    sigma, omega = O.kenney_laub(16, c)
    v = si.gaussian_field(d["dims"], 25)
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=12, tol=1e-12) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        y, rep = ctx.apply(torch.from_numpy(v).cuda(), adjoint=True)
        y = y.cpu().numpy()
    yo, _, _ = O.fom_lr(d["dims"], d["U"], v, -d["mu"], sigma, omega, k=12, tol=1e-12,
                        R=d["L"], L=d["R"], lam=np.conj(d["lam"]))
    assert _rel(y, yo) < TOL_FP64


def test_edge_cases(small):
    d = small
    sigma, omega = O.kenney_laub(6, 0.5)
    n = d["A"].shape[0]
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=10, tol=1e-12) as ctx:
        # b = 0 gives x = 0
        x, rep = ctx.apply(torch.zeros(n, dtype=torch.complex128, device="cuda"))
        assert rep["status"] == 0 and float(x.abs().max()) == 0.0
        # b inside the deflated subspace: x = x_P exactly, no Krylov work
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        bP = d["R"] @ np.arange(1, 7)
        x, rep = ctx.apply(torch.from_numpy(bP).cuda())
        xP = d["R"] @ (np.sign(d["lam"].real) * np.arange(1, 7))
        assert _rel(x.cpu().numpy(), xP) < 1e-10
        # b an eigenvector of A (no deflation): the Krylov space of A^2 has dimension 1,
        # Arnoldi breaks down in the first step and FOM is exact: x = g(lambda) b
        ctx.set_deflation(None, None, None)
        w, X, _ = O.eig(d["A"])
        j = int(np.argmax(np.abs(w)))
        bev = X[:, j]
        x, rep = ctx.apply(torch.from_numpy(bev).cuda())
        assert rep["breakdown"] == 1 and rep["status"] == 0
        g = w[j] * np.sum(omega / (w[j] ** 2 - sigma))
        assert _rel(x.cpu().numpy(), g * bev) < 1e-10


@pytest.mark.parametrize("adjoint", [False, True])
def test_split_form_matches_dense_target(lattice4, adjoint):
    """The split form (2s systems (A -+ a_i) in the Krylov space of A, weights omega_i/2)
    computes the same deflated rational function as the A^2 form: both match the dense
    target to the solve tolerance, the split form with k A-applications per cycle."""
    import paper_0910_2927_gb300 as pkg
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    b = np.stack([d["b"], si.gaussian_field(d["dims"], 77)])
    mu = -d["mu"] if adjoint else d["mu"]
    A = O.dense_hw(d["dims"], d["U"], mu)
    R, L, lam = (d["L"], d["R"], np.conj(d["lam"])) if adjoint else (d["R"], d["L"], d["lam"])
    with _ctx(d["dims"], d["U"], d["mu"], sigma, omega, k=30, tol=1e-12) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_formulation(pkg.FORM_A)
        x, rep = ctx.apply(torch.from_numpy(b).cuda(), adjoint=adjoint)
        x = x.cpu().numpy()
        assert rep["status"] == 0 and rep["matvecs"] == 30 * rep["cycles"]
        with pytest.raises(pkg.SignError):       # no per-shift iterates in the split form
            ctx.apply(torch.from_numpy(b).cuda(), shifts=True)
        ctx.set_precision(pkg.PREC_MIXED, 1e-8)
        with pytest.raises(pkg.SignError):       # FP64 form only
            ctx.apply(torch.from_numpy(b).cuda())
    for r in range(2):
        xstar = O.deflated_target(A, b[r], sigma, omega, R, L, lam)
        assert _rel(x[r], xstar) < 1e-9
