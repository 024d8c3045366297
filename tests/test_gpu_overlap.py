"""GPU parity of the overlap operator D_ov = 1 + gamma5 F(A), F the deflated rational
sign function (Sec. 1 with Algorithm 1), and of its inversion by restarted GMRES with
one batched sign solve per step: against the dense operator of the oracle's
eigendecomposition on the 4^4 configuration."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dense_overlap(d, sigma, omega):
    """I + gamma5 F(A), F the deflated rational sign function with the fixture's m pairs."""
    F = O.deflated_sign_matrix(d["A"], sigma, omega, m=len(d["lam"]), decomposition=d["eig"])
    return O.overlap_dense(F, int(np.prod(d["dims"])))


def test_overlap_apply_and_solve(lattice4):
    import paper_0910_2927_gb300 as pkg
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    D = _dense_overlap(d, sigma, omega)
    b = np.stack([d["b"], si.gaussian_field(d["dims"], 91)])
    with pkg.SignContext(d["dims"], mu=d["mu"]) as ctx:
        ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=30, tol=1e-13, max_cycles=2000)
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        y = ctx.overlap(torch.from_numpy(b).cuda()).cpu().numpy()
        x, its, rr = ctx.overlap_solve(torch.from_numpy(b).cuda(), tol=1e-10, k=20, max_restarts=40)
        x = x.cpu().numpy()
        with pytest.raises(pkg.SignError):
            ctx.overlap_solve(torch.from_numpy(b).cuda(), k=65)
    for r in range(2):
        yr = D @ b[r]
        assert np.linalg.norm(y[r] - yr) < 1e-10 * np.linalg.norm(yr)
        xr = np.linalg.solve(D, b[r])
        assert np.linalg.norm(D @ x[r] - b[r]) < 2e-10 * np.linalg.norm(b[r])
        assert np.linalg.norm(x[r] - xr) < 1e-7 * np.linalg.norm(xr)
    assert rr <= 1e-10 and its > 0


def test_overlap_apply_mixed_form(lattice4):
    """D_ov b through the mixed form (FP32 Krylov basis and stencil, FP64 refinement to 1e-9)
    agrees with the dense operator to the refinement's accuracy."""
    import paper_0910_2927_gb300 as pkg
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    D = _dense_overlap(d, sigma, omega)
    b = np.stack([d["b"], si.gaussian_field(d["dims"], 92), si.gaussian_field(d["dims"], 93)])
    with pkg.SignContext(d["dims"], mu=d["mu"]) as ctx:
        ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=30, tol=1e-10, max_cycles=2000)
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_precision(pkg.PREC_MIXED, 1e-9)
        y = ctx.overlap(torch.from_numpy(b).cuda()).cpu().numpy()
    for r in range(3):
        yr = D @ b[r]
        assert np.linalg.norm(y[r] - yr) < 1e-7 * np.linalg.norm(yr)
