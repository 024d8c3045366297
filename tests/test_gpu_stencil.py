"""GPU parity of the Wilson kernel H_W(mu) = gamma5 D_W(mu) against the oracle.

Element-by-element comparison on seeded random SU(3) fields; lattices with a
ragged site count (not a multiple of any CTA tile) and several fields."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(dims, U, mu, ap=(0, 0, 0, 1)):
    import paper_0910_2927_gb300 as pkg
    ctx = pkg.SignContext(dims, mu=mu, antiperiodic=ap)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    return ctx


@pytest.mark.parametrize("dims,ap", [((3, 4, 5, 6), (0, 0, 0, 1)), ((4, 4, 4, 4), (0, 0, 0, 1)),
                                     ((5, 2, 3, 7), (1, 1, 0, 1)), ((2, 2, 2, 2), (0, 0, 0, 0))])
@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0])
def test_fp64_stencil_matches_oracle(dims, ap, mu):
    U = si.random_su3_links(dims, 0.7, 11)
    nrhs = 3
    b = si.gaussian_block(dims, nrhs, 12)
    with _ctx(dims, U, mu, ap) as ctx:
        out = ctx.hw(torch.from_numpy(b).cuda()).cpu().numpy()
        outa = ctx.hw(torch.from_numpy(b).cuda(), adjoint=True).cpu().numpy()
    for r in range(nrhs):
        ref = O.hw(dims, U, b[r], mu, -1.6, ap)
        np.testing.assert_allclose(out[r], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        refa = O.hw(dims, U, b[r], -mu, -1.6, ap)
        np.testing.assert_allclose(outa[r], refa, rtol=0, atol=1e-13 * np.abs(refa).max())


@pytest.mark.parametrize("links", ["fp32", "bf16"])
def test_fp32_stencil_matches_oracle(links):
    import paper_0910_2927_gb300 as pkg
    dims, mu = (3, 4, 5, 6), 0.3
    U = si.random_su3_links(dims, 0.7, 13)
    b = si.gaussian_block(dims, 12, 14)
    with _ctx(dims, U, mu) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_BF16 if links == "bf16" else pkg.LINKS_FP32)
        out = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED).cpu().numpy()
    # error model: FP32 rounding of inputs and ~50 accumulated terms per entry;
    # BF16 links carry a relative rounding of 2^-9 per entry.
    tol = 2e-6 if links == "fp32" else 2e-2
    for r in range(12):
        ref = O.hw(dims, U, b[r], mu)
        err = np.linalg.norm(out[r] - ref) / np.linalg.norm(ref)
        assert err < tol, err


def test_stencil_skips_nothing_on_many_fields():
    """16 fields (more than one field block per CTA) all match."""
    dims, mu = (4, 3, 4, 5), 0.4
    U = si.random_su3_links(dims, 0.7, 15)
    b = si.gaussian_block(dims, 16, 16)
    with _ctx(dims, U, mu) as ctx:
        out = ctx.hw(torch.from_numpy(b).cuda()).cpu().numpy()
    for r in range(16):
        ref = O.hw(dims, U, b[r], mu)
        np.testing.assert_allclose(out[r], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_inner_products_match_numpy():
    """sgn_inner_products (Gram-Schmidt / projection coefficients) against numpy in FP64."""
    dims = (3, 4, 5, 6)
    U = si.random_su3_links(dims, 0.7, 17)
    V = si.gaussian_block(dims, 9, 18)
    w = si.gaussian_block(dims, 3, 19)
    with _ctx(dims, U, 0.3) as ctx:
        got = ctx.inner_products(torch.from_numpy(V).cuda(), torch.from_numpy(w).cuda())
    ref = w @ V.conj().T
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
