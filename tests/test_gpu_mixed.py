"""GPU parity of the mixed form: FP32 stencil and basis, FP64 scalars, refinement.

Bar: relative 2-norm error <= 1e-8 against the FP64 oracle (run to 1e-12)."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_MIXED = 1e-8


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def small():
    dims, mu = (3, 4, 3, 4), 0.3   # n = 1728
    U = si.random_su3_links(dims, 0.7, 41)
    A = O.dense_hw(dims, U, mu)
    R, L, lam, nxt = O.critical_eigenpairs(A, 8, extra=2)
    return dict(dims=dims, mu=mu, U=U, A=A, R=R, L=L, lam=lam, nxt=nxt)


@pytest.mark.parametrize("links", ["fp32", "bf16", "fp16"])
def test_mixed_matches_oracle(small, links):
    import paper_0910_2927_gb300 as pkg
    d = small
    c = O.scale_from_bounds(abs(d["nxt"][0]), 6.5)
    sigma, omega = O.kenney_laub(20, c)
    b = si.gaussian_block(d["dims"], 3, 42)
    with pkg.SignContext(d["dims"], mu=d["mu"]) as ctx:
        ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=16, tol=1e-10, max_cycles=2000)
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, {"fp32": pkg.LINKS_FP32, "bf16": pkg.LINKS_BF16,
                                                 "fp16": pkg.LINKS_FP16}[links])
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        x = x.cpu().numpy()
    assert rep["status"] == 0 and rep["err_est"] <= 1e-10, rep
    for r in range(3):
        xo, _, _ = O.fom_lr(d["dims"], d["U"], b[r], d["mu"], sigma, omega, k=16, tol=1e-12, max_cycles=5000,
                            R=d["R"], L=d["L"], lam=d["lam"])
        assert _rel(x[r], xo) < TOL_MIXED


def test_mixed_point_sources_config1(lattice4):
    """12 spin-colour point sources at 4^4 in one batched mixed solve."""
    import paper_0910_2927_gb300 as pkg
    d = lattice4
    c = O.scale_from_bounds(abs(d["lam_next"][0]), 6.0)
    sigma, omega = O.kenney_laub(16, c)
    b = si.point_sources(d["dims"], 12)
    with pkg.SignContext(d["dims"], mu=d["mu"]) as ctx:
        ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=30, tol=1e-10, max_cycles=2000)
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_precision(pkg.PREC_MIXED, 1e-8)
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        x = x.cpu().numpy()
    assert rep["status"] == 0, rep
    for r in (0, 5, 11):
        xo, _, _ = O.fom_lr(d["dims"], d["U"], b[r], d["mu"], sigma, omega, k=30, tol=1e-12, R=d["R"],
                            L=d["L"], lam=d["lam"])
        assert _rel(x[r], xo) < TOL_MIXED


@pytest.mark.parametrize("k_refine,batch", [(4, 5), (24, 0), (0, 7)])
def test_mixed_refinement_settings(small, k_refine, batch):
    """The correction solves' restart length and batch size change the work,
    not the result: every setting meets the tolerance and the oracle's x."""
    import paper_0910_2927_gb300 as pkg
    d = small
    c = O.scale_from_bounds(abs(d["nxt"][0]), 6.5)
    sigma, omega = O.kenney_laub(12, c)
    b = si.gaussian_block(d["dims"], 2, 43)
    with pkg.SignContext(d["dims"], mu=d["mu"]) as ctx:
        ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=16, tol=1e-10, max_cycles=2000)
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_precision(pkg.PREC_MIXED, 1e-8)
        ctx.set_refinement(k_refine, batch)
        x, rep = ctx.apply(torch.from_numpy(b).cuda())
        x = x.cpu().numpy()
    assert rep["status"] == 0 and rep["err_est"] <= 1e-10, rep
    for r in range(2):
        xo, _, _ = O.fom_lr(d["dims"], d["U"], b[r], d["mu"], sigma, omega, k=16, tol=1e-12, max_cycles=5000,
                            R=d["R"], L=d["L"], lam=d["lam"])
        assert _rel(x[r], xo) < TOL_MIXED


def test_refinement_setting_errors():
    import paper_0910_2927_gb300 as pkg
    with pkg.SignContext((2, 2, 2, 2)) as ctx:
        with pytest.raises(pkg.SignError):
            ctx.set_refinement(65, 0)
        with pytest.raises(pkg.SignError):
            ctx.set_refinement(8, -1)
