"""sgn_inner_products_noalloc: the allocation-free inner products, for callers that
cannot allocate device memory (frameworks that own every device allocation, loops
that must not pay for cudaMalloc).  Checked against sgn_inner_products.

Kept in its own file, collected last, so a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(lib, V, w, stream):
    J, n = V.shape
    out = torch.empty((w.shape[0], J), dtype=torch.complex128, device="cuda")
    rc = lib.sgn_inner_products_noalloc(C.c_void_p(V.data_ptr()), J, C.c_void_p(w.data_ptr()), n, w.shape[0],
                                        C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.sgn_last_error().decode()
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    import paper_0910_2927_gb300 as pkg
    lib = pkg.lib()
    dims = (6, 5, 4, 7)   # n = 10080 complex: 10 partial blocks per column, ragged tail
    U = si.random_su3_links(dims, 0.7, 61)
    stream = torch.cuda.current_stream()
    with pkg.SignContext(dims, mu=0.3) as ctx:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        for call, (J, nrhs, seed) in enumerate([(17, 5, 62), (40, 12, 63)]):
            V = torch.from_numpy(si.gaussian_block(dims, J, seed)).cuda()
            w = torch.from_numpy(si.gaussian_block(dims, nrhs, seed + 100)).cuda()
            got = _noalloc(lib, V, w, stream)
            ref = ctx.inner_products(V, w)
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= 1e-12 * scale, f"call {call}"


def test_noalloc_rejects_oversized_requests():
    import paper_0910_2927_gb300 as pkg
    lib = pkg.lib()
    n = 12 * 24 ** 4                      # 3888 partial blocks per column
    V = torch.zeros((1, 2), dtype=torch.complex128, device="cuda")   # never read: rejected first
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    rc = lib.sgn_inner_products_noalloc(C.c_void_p(V.data_ptr()), 64, C.c_void_p(V.data_ptr()), n, 12,
                                        C.c_void_p(out.data_ptr()), None)
    assert rc == 1   # SGN_ERR_ARG
    assert b"exceeds the fixed scratch" in lib.sgn_last_error()
