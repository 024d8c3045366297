"""The 8^4 workload on the GPU (n = 49,152): spread 0.7, s = 20 Kenney-Laub poles (eq. 6.2), restart
length k = 40, m = 20 deflated eigenpairs from the GPU eigensolver, at mu = 0 (Hermitian A) and 0.3;
and the mu = 1.0 regime (strongly non-Hermitian: without deflation restarted FOM diverges, the shifted
Hessenbergs of Algorithm 1 coming close to Ritz values) with the same parameters on the 4^4 lattice,
where the oracle's dense eigendecomposition supplies the 20 critical eigenpairs.

For each mu at 8^4:
* the deflation data are eigenpairs of the oracle's stencil (A r = lambda r, A^dag l = conj(lambda) l)
  with L^dag R = I, so that they are valid inputs for the oracle;
* the FP64 form (tol 1e-12) matches the oracle's FP64 FOM-LR with the same R, L, Lambda, shifts and
  weights to relative error <= 1e-10, in the same number of restart cycles (to one);
* the mixed form (FP32 stencil and basis, FP64 scalars, refinement, target 1e-8) matches it to 1e-8;
* at mu = 0 the GPU's Hessenberg matrix H_k of the Arnoldi relation (eq. 2.4) on the Hermitian A^2 is
  tridiagonal and Hermitian up to rounding, and the deflated eigenvalues are real."""
import math

import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS, S, K, M, EXTRA = (8, 8, 8, 8), 20, 40, 20, 4


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def inputs():
    g_seed, b_seed, _ = si.CONFIG_SEEDS[2]
    return si.random_su3_links(DIMS, 0.7, g_seed), si.gaussian_field(DIMS, b_seed)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_8x4_fp64_and_mixed_forms_match_oracle(inputs, mu):
    import paper_0910_2927_gb300 as pkg
    U, b = inputs
    with pkg.SignContext(DIMS, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        lam_all = ctx.build_deflation(M, extra=EXTRA, eig_tol=1e-10)
        b_max = abs(4.0 - 1.6) + 3.0 * math.sqrt(2.0) + math.sqrt(2.0 * math.cosh(2.0 * mu))
        c = 1.0 / math.sqrt(abs(lam_all[M]) * b_max)
        sigma, omega = pkg.kenney_laub(S, c)
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=K, tol=1e-12, max_cycles=3000)
        bd = torch.from_numpy(b).cuda()
        x64, rep64 = ctx.apply(bd)
        H, kk = ctx.hessenberg(0)
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        ctx.set_restart(k=K, tol=1e-10, max_cycles=3000)
        xm, repm = ctx.apply(bd)
        R, L, lam = ctx.get_deflation()
    x64, xm = x64.cpu().numpy(), xm.cpu().numpy()
    assert rep64["status"] == 0 and repm["status"] == 0
    # the deflation data satisfy eq. (4.1) for the oracle's operator
    for j in (0, M // 2, M - 1):
        rr = O.hw(DIMS, U, R[:, j], mu) - lam[j] * R[:, j]
        assert np.linalg.norm(rr) <= 1e-8 * abs(lam[j]) * np.linalg.norm(R[:, j])
        rl = O.hw(DIMS, U, L[:, j], -mu) - np.conj(lam[j]) * L[:, j]
        assert np.linalg.norm(rl) <= 1e-8 * abs(lam[j]) * np.linalg.norm(L[:, j])
    assert np.linalg.norm(L.conj().T @ R - np.eye(M)) < 1e-9
    assert np.all(np.abs(lam) <= np.abs(lam_all[M]))
    xo, orep, _ = O.fom_lr(DIMS, U, b, mu, sigma, omega, k=K, tol=1e-12, max_cycles=3000, R=R, L=L, lam=lam)
    assert orep["converged"]
    assert abs(orep["cycles"] - rep64["cycles"]) <= 1, (orep["cycles"], rep64["cycles"])
    assert _rel(x64, xo) <= 1e-10
    assert _rel(xm, xo) <= 1e-8
    if mu == 0.0:
        assert np.abs(lam.imag).max() <= 1e-10 * np.abs(lam).max()
        hmax = np.abs(H[:kk + 1, :kk]).max()
        upper = np.triu(H[:kk, :kk], 2)
        assert np.abs(upper).max() <= 1e-12 * hmax
        sub = np.diagonal(H[:kk, :kk], -1)
        sup = np.diagonal(H[:kk, :kk], 1)
        assert np.abs(sup - sub.conj()).max() <= 1e-12 * hmax
        assert np.abs(np.diagonal(H[:kk, :kk]).imag).max() <= 1e-12 * hmax


def test_mu1_regime_with_oracle_eigenpairs():
    """mu = 1.0, spread 0.7, s = 20, k = 40, m = 20 on the 4^4 lattice.  The oracle's dense
    eigendecomposition gives the deflation data (the 20 eigenpairs of smallest |lambda|, L^dag R = I).
    The GPU's FP64 form matches the oracle's FOM-LR to 1e-10 and the dense deflated target to 1e-9,
    the mixed form to 1e-8; and the GPU eigensolver (which needs its shift-invert route here: the
    unwanted eigenvalues of A^2 lie on three sides of the wanted ones) finds the same eigenvalues."""
    import paper_0910_2927_gb300 as pkg
    dims, mu = (4, 4, 4, 4), 1.0
    g_seed, b_seed, _ = si.CONFIG_SEEDS[2]
    U = si.random_su3_links(dims, 0.7, g_seed)
    b = si.gaussian_field(dims, b_seed)
    A = O.dense_hw(dims, U, mu)
    dec = O.eig(A)
    R, L, lam, nxt = O.critical_eigenpairs(A, M, extra=EXTRA, decomposition=dec)
    b_max = abs(4.0 - 1.6) + 3.0 * math.sqrt(2.0) + math.sqrt(2.0 * math.cosh(2.0 * mu))
    sigma, omega = O.kenney_laub(S, 1.0 / math.sqrt(abs(nxt[0]) * b_max))
    xo, orep, _ = O.fom_lr(dims, U, b, mu, sigma, omega, k=K, tol=1e-12, max_cycles=3000, R=R, L=L, lam=lam)
    assert orep["converged"]
    target = O.deflated_target(A, b, sigma, omega, R=R, L=L, lam=lam)
    with pkg.SignContext(dims, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=K, tol=1e-12, max_cycles=3000)
        ctx.set_deflation(R, L, lam)
        bd = torch.from_numpy(b).cuda()
        x64, rep64 = ctx.apply(bd)
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        ctx.set_restart(k=K, tol=1e-10, max_cycles=3000)
        xm, repm = ctx.apply(bd)
        lam_gpu = ctx.build_deflation(M, extra=EXTRA, eig_tol=1e-10)
    x64, xm = x64.cpu().numpy(), xm.cpu().numpy()
    assert rep64["status"] == 0 and repm["status"] == 0
    assert _rel(x64, xo) <= 1e-10
    assert _rel(x64, target) <= 1e-9
    assert _rel(xm, xo) <= 1e-8
    # No cycle-count comparison here: in this slowly converging non-normal regime the
    # residual estimate oscillates around the tolerance for many cycles, and rounding alone
    # (the oracle's OpenMP sums) moved its stopping cycle from 183 to 299 between two runs
    # while x agreed to 1e-10 both times.
    ref = np.concatenate([lam, nxt[:EXTRA]])
    for z in lam_gpu:
        assert np.min(np.abs(ref - z)) <= 1e-9 * abs(z), z
