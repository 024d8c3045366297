"""Error statuses of the C ABI, each provoked on the host side (no GPU fault, no device trap):

* calls out of order (apply before load_gauge) -> SGN_ERR_STATE;
* deflation data dropped by a change of the operator (mu, kernel mass, boundary, gauge field):
  every solve refuses with SGN_ERR_STATE until the data are built, set or cleared (Sec. 4: R, L,
  Lambda are eigenpairs of one operator, eq. (4.1));
* NaN in host b, in host links, and in device b (met inside the iteration) -> SGN_ERR_NONFINITE;
* an eigenvalue with Re lambda = 0 (sign undefined) -> SGN_ERR_DEFLATION;
* an ambiguous selection |lambda_m| = |lambda_m+1| (colour-degenerate free field) -> SGN_ERR_DEFLATION;
* a shift on a Ritz value: a singular shifted Hessenberg system (H_k - sigma) -> SGN_ERR_BREAKDOWN;

and determinism: the same solve twice gives bitwise equal results (fixed-order reductions,
no atomics in any sum)."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OK, ERR_ARG, ERR_BREAKDOWN, ERR_DEFLATION, ERR_NONFINITE, ERR_STATE = 0, 1, 4, 5, 6, 8


def _pkg():
    import paper_0910_2927_gb300 as pkg
    return pkg


def _code(fn, *args):
    pkg = _pkg()
    with pytest.raises(pkg.SignError) as ei:
        fn(*args)
    return ei.value.code


@pytest.fixture(scope="module")
def small():
    dims, mu = (3, 2, 3, 4), 0.3
    U = si.random_su3_links(dims, 0.7, 21)
    A = O.dense_hw(dims, U, mu)
    R, L, lam, _ = O.critical_eigenpairs(A, 6, extra=2)
    return dict(dims=dims, mu=mu, U=U, R=R, L=L, lam=lam, b=si.gaussian_block(dims, 2, 22))


def _ctx(d, mu=None):
    pkg = _pkg()
    ctx = pkg.SignContext(d["dims"], mu=d["mu"] if mu is None else mu)
    ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
    sigma, omega = O.kenney_laub(12, 0.4)
    ctx.set_rational(sigma, omega)
    ctx.set_restart(k=10, tol=1e-10, max_cycles=500)
    return ctx


def test_apply_before_load_gauge_is_a_state_error(small):
    pkg = _pkg()
    with pkg.SignContext(small["dims"], mu=0.3) as ctx:
        ctx.set_rational(*O.kenney_laub(4, 0.5))
        b = torch.from_numpy(small["b"]).cuda()
        assert _code(ctx.apply, b) == ERR_STATE
        assert _code(ctx.hw, b) == ERR_STATE
        assert _code(ctx.build_deflation, 2) == ERR_STATE


def test_apply_before_rational_function_is_a_state_error(small):
    pkg = _pkg()
    with pkg.SignContext(small["dims"], mu=0.3) as ctx:
        ctx.load_gauge(torch.from_numpy(small["U"]).cuda())
        assert _code(ctx.apply, torch.from_numpy(small["b"]).cuda()) == ERR_STATE


@pytest.mark.parametrize("change", ["mu", "mass", "boundary", "gauge"])
def test_operator_change_makes_deflation_stale(small, change):
    """After the operator changes, the old R, L, Lambda are not its eigenpairs: every solve
    refuses until new data are set (or m = 0 is chosen), instead of running undeflated."""
    d = small
    b = torch.from_numpy(d["b"]).cuda()
    with _ctx(d) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        x0, rep = ctx.apply(b)
        assert rep["status"] == OK
        if change == "mu":
            ctx.set_mu(d["mu"] + 0.1)
        elif change == "mass":
            ctx.set_kernel_mass(-1.5)
        elif change == "boundary":
            ctx.set_boundary((0, 0, 0, 0))
        else:
            ctx.load_gauge(torch.from_numpy(d["U"]).cuda())
        assert ctx.m == 0
        assert _code(ctx.apply, b) == ERR_STATE
        assert _code(ctx.apply, d["b"]) == ERR_STATE          # host-buffer path as well
        assert _code(ctx.overlap, b) == ERR_STATE
        assert _code(ctx.apply_direct, b, 8) == ERR_STATE
        lib = _pkg().lib()
        out = np.zeros(2)
        bb = b.contiguous()
        rc = lib.sgn_grad_mu(ctx._h, C.c_void_p(bb.data_ptr()), C.c_void_p(bb.data_ptr()), 2, out.ctypes.data)
        assert rc == ERR_STATE
        # an explicit choice of no deflation lifts the refusal
        ctx.set_deflation(None, None, None)
        _, rep = ctx.apply(b)
        assert rep["status"] == OK


def test_same_mu_keeps_deflation(small):
    d = small
    with _ctx(d) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_mu(d["mu"])
        assert ctx.m == 6
        _, rep = ctx.apply(torch.from_numpy(d["b"]).cuda())
        assert rep["status"] == OK


def test_setting_new_deflation_after_change_works(small):
    d = small
    mu2 = d["mu"] + 0.2
    A2 = O.dense_hw(d["dims"], d["U"], mu2)
    R2, L2, lam2, _ = O.critical_eigenpairs(A2, 6, extra=2)
    sigma, omega = O.kenney_laub(12, 0.4)
    with _ctx(d) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        ctx.set_mu(mu2)
        ctx.set_deflation(R2, L2, lam2)
        x, rep = ctx.apply(torch.from_numpy(d["b"][0]).cuda())
        assert rep["status"] == OK
    ref = O.deflated_target(A2, d["b"][0], sigma, omega, R=R2, L=L2, lam=lam2)
    assert np.linalg.norm(x.cpu().numpy() - ref) < 1e-8 * np.linalg.norm(ref)


def test_signapply_refuses_silent_mu_change(small):
    """SignApply at another mu than the context's, with deflation data present, raises unless
    the context was told to rebuild them (it then runs deflated at the new mu)."""
    from paper_0910_2927_gb300.autograd import SignApply
    d = small
    bt = torch.from_numpy(d["b"][0]).cuda()
    with _ctx(d) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        with pytest.raises(ValueError):
            SignApply.apply(bt, torch.tensor(d["mu"] + 0.1, dtype=torch.float64), ctx)
        assert ctx.m == 6 and ctx.mu == d["mu"]
        # set, not built: there is nothing to rebuild from
        ctx.rebuild_deflation_on_mu_change = True
        with pytest.raises(ValueError):
            SignApply.apply(bt, torch.tensor(d["mu"] + 0.1, dtype=torch.float64), ctx)


def test_signapply_rebuilds_deflation_when_asked(small):
    from paper_0910_2927_gb300.autograd import SignApply
    d = small
    mu2 = d["mu"] + 0.1
    with _ctx(d) as ctx:
        lam = ctx.build_deflation(4, extra=2, eig_tol=1e-11)
        ctx.rebuild_deflation_on_mu_change = True
        x = SignApply.apply(torch.from_numpy(d["b"][0]).cuda(), torch.tensor(mu2, dtype=torch.float64), ctx)
        assert ctx.mu == mu2 and ctx.m == 4
        R, L, lam2 = ctx.get_deflation()
    # the rebuilt pairs are eigenpairs of the operator at the new mu (oracle stencil)
    for j in range(4):
        res = O.hw(d["dims"], d["U"], R[:, j], mu2) - lam2[j] * R[:, j]
        assert np.linalg.norm(res) < 1e-8 * abs(lam2[j]) * np.linalg.norm(R[:, j])
    assert np.isfinite(x.detach().cpu().numpy()).all()


def test_nonfinite_inputs(small):
    d = small
    pkg = _pkg()
    bad = d["b"].copy()
    bad[1, 17] = np.nan
    with _ctx(d) as ctx:
        assert _code(ctx.apply, bad) == ERR_NONFINITE                          # host b, checked on entry
        lib = pkg.lib()
        bd = torch.from_numpy(bad).cuda()
        xd = torch.empty_like(bd)
        rep = pkg.Report()
        rc = lib.sgn_apply(ctx._h, C.c_void_p(bd.data_ptr()), C.c_void_p(xd.data_ptr()), 2, 0, C.byref(rep))
        assert rc == ERR_NONFINITE, lib.sgn_last_error().decode()              # device b: met in the iteration
        # the context stays usable
        _, rep2 = ctx.apply(torch.from_numpy(d["b"]).cuda())
        assert rep2["status"] == OK
    Ubad = d["U"].copy()
    Ubad[5, 2, 1, 1] = np.inf
    with pkg.SignContext(d["dims"], mu=0.3) as ctx:
        assert _code(ctx.load_gauge, Ubad) == ERR_NONFINITE                    # host links


def test_eigenvalue_on_imaginary_axis_is_rejected(small):
    d = small
    lam = d["lam"].copy()
    lam[2] = 1j * abs(lam[2])
    with _ctx(d) as ctx:
        assert _code(ctx.set_deflation, d["R"], d["L"], lam) == ERR_DEFLATION


def test_ambiguous_selection_is_rejected():
    """Free field (U = 1): every eigenvalue of H_W is (at least) three-fold degenerate in colour,
    so the m = 1 smallest |lambda| cannot be told apart from the next one."""
    pkg = _pkg()
    dims = (4, 2, 2, 4)
    U = np.zeros((int(np.prod(dims)), 4, 3, 3), dtype=np.complex128)
    U[:, :, range(3), range(3)] = 1.0
    with pkg.SignContext(dims, mu=0.0) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        with pytest.raises(pkg.SignError) as ei:
            ctx.build_deflation(1, extra=2, eig_tol=1e-10)
        assert ei.value.code == ERR_DEFLATION
        assert "coincide" in str(ei.value)


def test_shift_on_ritz_value_is_a_breakdown():
    """Exact arithmetic by construction: free field, m_W = -2, periodic, mu = 0.  A constant
    spinor u with one unit component is an eigenvector, D_W u = (4 + m_W - 4) u = -2 u, so
    A^2 u = 4 u with every value a power of two: the first Arnoldi step gives H_1 = [4] exactly and
    meets the invariant subspace.  The shift sigma = 4 makes H_1 - sigma exactly singular."""
    pkg = _pkg()
    dims = (2, 2, 2, 2)
    vol = 16
    U = np.zeros((vol, 4, 3, 3), dtype=np.complex128)
    U[:, :, range(3), range(3)] = 1.0
    b = np.zeros((vol, 12), dtype=np.complex128)
    b[:, 0] = 1.0
    with pkg.SignContext(dims, mu=0.0, mass=-2.0, antiperiodic=(0, 0, 0, 0)) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_rational(np.array([4.0]), np.array([1.0]))
        ctx.set_restart(k=4, tol=1e-12, max_cycles=3)
        with pytest.raises(pkg.SignError) as ei:
            ctx.apply(torch.from_numpy(b.reshape(-1)).cuda())
        assert ei.value.code == ERR_BREAKDOWN, str(ei.value)
        # a regular shift on the same operator solves exactly: x = A (A^2 - sigma)^{-1} b = -2 u / (4 - sigma)
        ctx.set_rational(np.array([-4.0]), np.array([1.0]))
        x, rep = ctx.apply(torch.from_numpy(b.reshape(-1)).cuda())
        assert rep["status"] == OK
        assert np.abs(x.cpu().numpy() - (-2.0 / 8.0) * b.reshape(-1)).max() < 1e-15


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solves_are_bitwise_repeatable(small, prec):
    pkg = _pkg()
    d = small
    b = torch.from_numpy(si.gaussian_block(d["dims"], 3, 31)).cuda()
    with _ctx(d) as ctx:
        ctx.set_deflation(d["R"], d["L"], d["lam"])
        if prec == "mixed":
            ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        x1, r1 = ctx.apply(b)
        x2, r2 = ctx.apply(b)
        x3, _ = ctx.apply(b.cpu().numpy())     # host-buffer path: same kernels, same result
    assert r1["cycles"] == r2["cycles"]
    assert torch.equal(x1, x2)
    assert np.array_equal(x1.cpu().numpy(), x3)
