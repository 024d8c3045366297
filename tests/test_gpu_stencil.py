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


LINK_STORAGE = {"fp32": 0, "bf16": 1, "fp16": 2}


@pytest.mark.parametrize("links", ["fp32", "bf16", "fp16"])
def test_fp32_stencil_matches_oracle(links):
    import paper_0910_2927_gb300 as pkg
    dims, mu = (3, 4, 5, 6), 0.3
    U = si.random_su3_links(dims, 0.7, 13)
    b = si.gaussian_block(dims, 12, 14)
    with _ctx(dims, U, mu) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, LINK_STORAGE[links])
        out = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED).cpu().numpy()
    # error model: FP32 rounding of inputs and ~50 accumulated terms per entry;
    # BF16 links carry a relative rounding of up to 2^-9 per entry, FP16 links 2^-12.
    tol = {"fp32": 2e-6, "bf16": 2e-2, "fp16": 3e-3}[links]
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


def test_packed_layout_roundtrip_and_stencil():
    """pack/unpack invert each other, the packed order is the documented one
    (entry k of site s at (k/2) 2V + 2s + k%2), and the stencil on packed
    fields equals the packed result of the stencil on natural fields."""
    import paper_0910_2927_gb300 as pkg
    dims, mu = (3, 4, 5, 6), 0.3
    vol = int(np.prod(dims))
    U = si.random_su3_links(dims, 0.7, 21)
    b = si.gaussian_block(dims, 5, 22)
    # the documented order, written out on the host
    nat = b.reshape(5, vol, 6, 2)
    want_packed = np.ascontiguousarray(nat.transpose(0, 2, 1, 3)).reshape(5, -1)
    with _ctx(dims, U, mu) as ctx:
        for prec, dt in ((pkg.PREC_FP64, np.complex128), (pkg.PREC_MIXED, np.complex64)):
            bd = torch.from_numpy(b.astype(dt)).cuda()
            pk = ctx.pack(bd, prec)
            assert np.array_equal(pk.cpu().numpy(), want_packed.astype(dt))
            assert torch.equal(ctx.unpack(pk, prec), bd)
            for adj in (False, True):
                direct = ctx.hw(pk, precision=prec, adjoint=adj, packed=True)
                via = ctx.pack(ctx.hw(bd, precision=prec, adjoint=adj), prec)
                assert torch.equal(direct, via)


@pytest.mark.parametrize("shape", ["32,4,3", "64,2,2", "32,2,3", "64,3,1", "128,1,2",
                                   "32,4,1,1", "64,2,2,1", "128,1,2,1", "256,1,1,1",
                                   "32,4,2,2", "64,2,2,2", "128,1,2,2", "256,1,2,2",
                                   "64,2,2,3", "128,1,2,3",
                                   "1,2,1,4", "2,4,1,4", "4,2,1,4", "8,1,1,4", "1,8,1,4"])
def test_fp32_stencil_launch_shapes(shape, monkeypatch):
    """Every launch shape (sites per CTA, thread rows, fields per thread, the kernel
    that stages neighbours through shared memory with cp.async, and the kernel with
    paired FP32 arithmetic over two fields) gives
    the oracle's result, including field counts that leave the last thread's
    group of fields ragged (5 fields, 2 or 3 per thread)."""
    import paper_0910_2927_gb300 as pkg
    monkeypatch.setenv("SGN_STENCIL_SHAPE", shape)
    dims, mu = (5, 2, 3, 7), 0.3
    U = si.random_su3_links(dims, 0.7, 31)
    b = si.gaussian_block(dims, 5, 32)
    with _ctx(dims, U, mu, (1, 1, 0, 1)) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        out = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED).cpu().numpy()
        outa = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED, adjoint=True).cpu().numpy()
    for r in range(5):
        ref = O.hw(dims, U, b[r], mu, -1.6, (1, 1, 0, 1))
        assert np.linalg.norm(out[r] - ref) / np.linalg.norm(ref) < 2e-6
        refa = O.hw(dims, U, b[r], -mu, -1.6, (1, 1, 0, 1))
        assert np.linalg.norm(outa[r] - refa) / np.linalg.norm(refa) < 2e-6


@pytest.mark.parametrize("shape", ["32,12,3", "64,2,1,2", "128,4,2,2", "64,2,3,3", "3,3,1,4", "2,2,2,4"])
def test_invalid_launch_shape_is_an_error(shape, monkeypatch):
    """A shape outside the kernel's limits (384 threads with 3 fields each; the paired
    kernel with one field per thread, or with 512 threads) is refused with an error."""
    import paper_0910_2927_gb300 as pkg
    monkeypatch.setenv("SGN_STENCIL_SHAPE", shape)
    dims = (4, 4, 4, 4)
    U = si.random_su3_links(dims, 0.7, 33)
    b = si.gaussian_block(dims, 12, 34)
    with _ctx(dims, U, 0.3) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        with pytest.raises(pkg.SignError):
            ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED)


@pytest.mark.parametrize("links", ["bf16", "fp16"])
@pytest.mark.parametrize("shape", ["64,2,2,1", "32,4,1,1", "64,2,2,2", "128,1,2,3", "2,4,1,4", "1,6,1,4",
                                   "64,4,1,0", "32,4,3,0"])
def test_low_precision_links_every_kernel_many_fields(shape, links, monkeypatch):
    """Every FP32 stencil kernel (one to three fields per thread, the shared-memory staged
    kernel, the paired kernel, the colour-split kernel) with BF16 or FP16 links and 13 fields
    (several CTAs per site tile) matches the oracle within the rounding of the links."""
    import paper_0910_2927_gb300 as pkg
    monkeypatch.setenv("SGN_STENCIL_SHAPE", shape)
    dims, mu = (4, 3, 4, 5), 0.4
    U = si.random_su3_links(dims, 0.7, 35)
    b = si.gaussian_block(dims, 13, 36)
    with _ctx(dims, U, mu) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, LINK_STORAGE[links])
        out = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED).cpu().numpy()
    tol = {"bf16": 2e-2, "fp16": 3e-3}[links]
    for r in (0, 6, 12):
        ref = O.hw(dims, U, b[r], mu)
        assert np.linalg.norm(out[r] - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("shape", ["1,4,1,4", "4,1,1,4"])
def test_colour_split_stencil_ragged_tail(shape, monkeypatch):
    """The colour-split kernel (10 sites per warp, three lanes per site) on a volume that
    leaves the last warp's group of sites ragged (135 sites), both hop directions."""
    import paper_0910_2927_gb300 as pkg
    monkeypatch.setenv("SGN_STENCIL_SHAPE", shape)
    dims, mu = (3, 3, 3, 5), 0.6
    U = si.random_su3_links(dims, 0.7, 37)
    b = si.gaussian_block(dims, 3, 38)
    with _ctx(dims, U, mu) as ctx:
        ctx.set_precision(pkg.PREC_MIXED, 1e-8, pkg.LINKS_FP32)
        out = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED).cpu().numpy()
        outa = ctx.hw(torch.from_numpy(b).cuda(), precision=pkg.PREC_MIXED, adjoint=True).cpu().numpy()
    for r in range(3):
        ref = O.hw(dims, U, b[r], mu)
        assert np.linalg.norm(out[r] - ref) / np.linalg.norm(ref) < 2e-6
        refa = O.hw(dims, U, b[r], -mu)
        assert np.linalg.norm(outa[r] - refa) / np.linalg.norm(refa) < 2e-6


@pytest.mark.parametrize("dims,ap", [((3, 4, 5, 6), (0, 0, 0, 1)), ((5, 2, 3, 7), (1, 1, 0, 1)),
                                     ((2, 2, 2, 2), (0, 0, 0, 0))])
@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0])
def test_float_float_stencil_matches_oracle(dims, ap, mu):
    """The float-float stencil (the mixed form's true residuals) against the oracle's FP64 stencil:
    within 1e-13 of the largest entry, like the FP64 stencil, on ragged lattices, both boundary
    conditions, both hop directions (adjoint), 3 fields (the last CTA's field pair ragged)."""
    U = si.random_su3_links(dims, 0.7, 11)
    b = si.gaussian_block(dims, 3, 12)
    with _ctx(dims, U, mu, ap) as ctx:
        out = ctx.hw(torch.from_numpy(b).cuda(), float_float=True).cpu().numpy()
        outa = ctx.hw(torch.from_numpy(b).cuda(), adjoint=True, float_float=True).cpu().numpy()
    for r in range(3):
        ref = O.hw(dims, U, b[r], mu, -1.6, ap)
        np.testing.assert_allclose(out[r], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        refa = O.hw(dims, U, b[r], -mu, -1.6, ap)
        np.testing.assert_allclose(outa[r], refa, rtol=0, atol=1e-13 * np.abs(refa).max())


def test_float_float_stencil_is_more_than_fp32():
    """Float-float is not FP32 in disguise: on inputs with low-order bits (x = 1 + 2^-30 u) the
    result keeps them (error 1e-13 against the FP32 stencil's 1e-7), and the flag is refused for
    complex64 fields."""
    import paper_0910_2927_gb300 as pkg
    dims, mu = (4, 3, 4, 5), 0.4
    U = si.random_su3_links(dims, 0.7, 51)
    b = si.gaussian_block(dims, 2, 52)
    x = 1.0 + 2.0 ** -30 * b
    with _ctx(dims, U, mu) as ctx:
        out = ctx.hw(torch.from_numpy(x).cuda(), float_float=True).cpu().numpy()
        with pytest.raises(pkg.SignError):
            ctx.hw(torch.from_numpy(x).cuda(), precision=pkg.PREC_MIXED, float_float=True)
    for r in range(2):
        ref = O.hw(dims, U, x[r], mu)
        assert np.linalg.norm(out[r] - ref) / np.linalg.norm(ref) < 1e-13
