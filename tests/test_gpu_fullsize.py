"""Parity at the benchmark's full sizes, in the benchmark's launch configuration, on outputs
the oracle can compute one by one.

* 10^4 lattice, spread 0.7, mu = 0.3, 12 spin-colour point sources, s = 20, k = 40, m = 30 (the
  default benchmark workload): the GPU eigensolver's deflation data satisfy the eigen-equations
  and L^dag R = I (checked with the oracle's C stencil), and the mixed-form batched solve at
  tol 1e-8 agrees on two sampled columns with the oracle's FP64 FOM-LR run with the same
  deflation data, shifts and weights.
* 24^4 lattice, spread 0.7, mu = 0.2, 12 columns (the stencil bandwidth workload): the tuned
  FP32 stencil and the FP64 stencil agree with the oracle's stencil on sampled sites, the
  boundary sites of every direction included."""
import math

import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_10x4_workload_deflation_and_mixed_solve():
    import paper_0910_2927_gb300 as pkg
    dims, mu, s, k, m = (10, 10, 10, 10), 0.3, 20, 40, 30
    U = si.random_su3_links(dims, 0.7, si.CONFIG_SEEDS[3][0])
    B = si.point_sources(dims, 12)
    with pkg.SignContext(dims, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        lam = ctx.build_deflation(m, extra=4, eig_tol=1e-9)
        b_max = abs(4.0 - 1.6) + 3.0 * math.sqrt(2.0) + math.sqrt(2.0 * math.cosh(2.0 * mu))
        c = 1.0 / math.sqrt(abs(lam[m]) * b_max)
        sigma, omega = pkg.kenney_laub(s, c)
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=k, tol=1e-8, max_cycles=2000)
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        x, rep = ctx.apply(torch.from_numpy(B).cuda())
        x = x.cpu().numpy()
        R, L, lamd = ctx.get_deflation()
    assert rep["status"] == 0 and R.shape == (12 * 10 ** 4, m)
    # eigen-equations with the oracle's stencil: A r = lambda r, A^dag l = conj(lambda) l
    # (set-up tolerance 1e-9 on the relative eigen-residual; a wrong pair is off by O(1))
    for j in (0, m // 2, m - 1):
        rr = O.hw(dims, U, R[:, j], mu) - lamd[j] * R[:, j]
        assert np.linalg.norm(rr) <= 1e-7 * abs(lamd[j]) * np.linalg.norm(R[:, j])
        rl = O.hw(dims, U, L[:, j], -mu) - np.conj(lamd[j]) * L[:, j]
        assert np.linalg.norm(rl) <= 1e-7 * abs(lamd[j]) * np.linalg.norm(L[:, j])
    assert np.linalg.norm(L.conj().T @ R - np.eye(m)) < 1e-8
    # sampled columns against the oracle's FP64 FOM-LR with the same deflation data
    for col in (0, 7):
        xo, orep, _ = O.fom_lr(dims, U, B[col], mu, sigma, omega, k=k, tol=1e-10, max_cycles=2000,
                               R=R, L=L, lam=lamd)
        assert orep["converged"]
        assert _rel(x[col], xo) < 1e-8


def test_24x4_stencil_sampled_sites():
    import paper_0910_2927_gb300 as pkg
    dims, mu = (24, 24, 24, 24), 0.2
    V = 24 ** 4
    U = si.random_su3_links(dims, 0.7, si.CONFIG_SEEDS[5][0])
    psi = si.gaussian_block(dims, 12, 501)
    rng = np.random.default_rng(502)
    # random sites and the sites on both faces of every direction through the origin's corner
    faces = [0, 23, 23 * 24, 23 * 24 ** 2, 23 * 24 ** 3, V - 1, 24 ** 3 - 1, 24 ** 2 * 23 + 23]
    sites = np.unique(np.concatenate([rng.choice(V, 256, replace=False), faces]))
    with pkg.SignContext(dims, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        dev = torch.from_numpy(psi).cuda()
        idx = torch.from_numpy(sites).cuda()
        out32 = ctx.hw(dev, precision=pkg.PREC_MIXED).reshape(12, V, 12)[:, idx, :].cpu().numpy()
        out64 = ctx.hw(dev[3:4], precision=pkg.PREC_FP64).reshape(V, 12)[idx, :].cpu().numpy()
    for col in (0, 5, 11):
        ref = O.hw_sites(dims, U, psi[col], sites, mu)
        assert _rel(out32[col], ref) < 2e-6
    ref3 = O.hw_sites(dims, U, psi[3], sites, mu)
    assert _rel(out64, ref3) < 1e-13


def test_24x4_solve_shifted_residuals_sampled():
    """The 24^4 lattice of the throughput workload (spread 0.7, mu = 0.2, s = 20, k = 40), one
    Gaussian column, FP64 form, undeflated (its 40-pair set-up takes minutes): every shifted
    system's residual b~ - (A^2 - sigma_i) x_i, with b~ = A b and A^2 applied by the oracle's stencil,
    is at the solver's tolerance on sampled sites and the sites on every face; and the returned x is
    sum_i omega_i x_i there (Algorithm 1's combination, eq. 2.3).  A wrong hop, sign, shift or weight
    gives O(1) residuals."""
    import paper_0910_2927_gb300 as pkg
    dims, mu, s, k, tol = (24, 24, 24, 24), 0.2, 20, 40, 1e-10
    V = 24 ** 4
    U = si.random_su3_links(dims, 0.7, si.CONFIG_SEEDS[5][0])
    b = si.gaussian_field(dims, si.CONFIG_SEEDS[5][1])
    b_max = abs(4.0 - 1.6) + 3.0 * math.sqrt(2.0) + math.sqrt(2.0 * math.cosh(2.0 * mu))
    sigma, omega = pkg.kenney_laub(s, 1.0 / math.sqrt(0.18 * b_max))
    with pkg.SignContext(dims, mu=mu) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_rational(sigma, omega)
        ctx.set_restart(k=k, tol=tol, max_cycles=3000)
        x, xs, rep = ctx.apply(torch.from_numpy(b).cuda(), shifts=True)
        x = x.cpu().numpy().reshape(V, 12)
        xs = xs[:, 0].cpu().numpy()
    assert rep["status"] == 0
    rng = np.random.default_rng(503)
    faces = [0, 23, 23 * 24, 23 * 24 ** 2, 23 * 24 ** 3, V - 1]
    sites = np.unique(np.concatenate([rng.choice(V, 96, replace=False), faces]))
    # sites whose A x is needed for A^2 x on `sites`: the sites and their 8 neighbours
    co = np.stack(np.unravel_index(sites, dims[::-1])[::-1], axis=1)   # (x, y, z, t)
    near = [sites]
    for d in range(4):
        for step in (1, -1):
            c2 = co.copy()
            c2[:, d] = (c2[:, d] + step) % 24
            near.append(np.ravel_multi_index(tuple(c2[:, ::-1].T), dims[::-1]))
    near = np.unique(np.concatenate(near))
    bt = O.hw_sites(dims, U, b, sites, mu)                        # b~ = A b on the sampled sites
    for i in (0, 7, s - 1):
        ax = np.zeros((V, 12), dtype=np.complex128)
        ax[near] = O.hw_sites(dims, U, xs[i], near, mu)            # A x_i where A^2 x_i needs it
        a2x = O.hw_sites(dims, U, ax.reshape(-1), sites, mu)
        r = bt - (a2x - sigma[i] * xs[i].reshape(V, 12)[sites])
        assert np.linalg.norm(r) <= 100 * tol * np.linalg.norm(bt), (i, np.linalg.norm(r) / np.linalg.norm(bt))
    comb = sum(omega[i] * xs[i].reshape(V, 12)[sites] for i in range(s))
    assert np.linalg.norm(comb - x[sites]) <= 1e-12 * np.linalg.norm(x[sites])
