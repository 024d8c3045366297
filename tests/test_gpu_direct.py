"""GPU parity of the direct projection of eq. (6.3), x = x_P + ||r|| V_k sign(H_k) e_1
(k Arnoldi steps on A, sign(H_k) by Roberts' Newton iteration), against the oracle's
direct_projection at the same k: plain and deflated, forward and adjoint, a ragged
lattice, and k = n, where the projection is exact and equals the dense sign(A) b."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ctx(dims, U, mu):
    import paper_0910_2927_gb300 as pkg
    ctx = pkg.SignContext(dims, mu=mu)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    return ctx


@pytest.mark.parametrize("adjoint", [False, True])
def test_direct_projection_deflated(adjoint):
    dims, mu, k = (3, 2, 3, 4), 0.3, 60   # n = 864: several tiles and a ragged tail
    U = si.random_su3_links(dims, 0.7, 21)
    A = O.dense_hw(dims, U, mu)
    R, L, lam, _ = O.critical_eigenpairs(A, 6, extra=2)
    b = np.stack([si.gaussian_field(dims, 22), si.gaussian_field(dims, 23)])
    with _ctx(dims, U, mu) as ctx:
        ctx.set_deflation(R, L, lam)
        x, ku = ctx.apply_direct(torch.from_numpy(b).cuda(), k, adjoint=adjoint)
    x = x.cpu().numpy()
    assert ku == k
    Aop = A.conj().T if adjoint else A
    Rop, Lop, lop = (L, R, lam.conj()) if adjoint else (R, L, lam)
    for r in range(2):
        ref = O.direct_projection(Aop, b[r], k, Rop, Lop, lop)
        assert _rel(x[r], ref) < 1e-10


def test_direct_projection_plain_and_exact_at_full_dimension():
    dims, mu = (2, 2, 2, 2), 0.4
    U = si.random_su3_links(dims, 0.6, 81)
    A = O.dense_hw(dims, U, mu)
    b = si.gaussian_field(dims, 82)
    n = A.shape[0]
    with _ctx(dims, U, mu) as ctx:
        x24, k24 = ctx.apply_direct(torch.from_numpy(b).cuda(), 24)
        xn, kn = ctx.apply_direct(torch.from_numpy(b).cuda(), n)
    assert k24 == 24 and kn <= n
    assert _rel(x24.cpu().numpy(), O.direct_projection(A, b, 24)) < 1e-10
    assert _rel(xn.cpu().numpy(), O.sign_eig(A) @ b) < 1e-9


def test_direct_projection_errors():
    import paper_0910_2927_gb300 as pkg
    dims = (2, 2, 2, 2)
    U = si.random_su3_links(dims, 0.6, 81)
    b = torch.from_numpy(si.gaussian_field(dims, 82)).cuda()
    with _ctx(dims, U, 0.4) as ctx:
        with pytest.raises(pkg.SignError):
            ctx.apply_direct(b, 0)
        with pytest.raises(pkg.SignError):
            ctx.apply_direct(b, 5000)


def test_direct_projection_zero_column_and_k1():
    """A zero column gives x = 0 (no Krylov work) beside a normal one; k = 1 is the
    one-dimensional projection x = ||b|| sign(h_11) v_1 with h_11 = v_1^dag A v_1."""
    dims, mu = (2, 2, 2, 3), 0.3
    U = si.random_su3_links(dims, 0.6, 83)
    A = O.dense_hw(dims, U, mu)
    b1 = si.gaussian_field(dims, 84)
    b = np.stack([np.zeros_like(b1), b1])
    with _ctx(dims, U, mu) as ctx:
        x, ku = ctx.apply_direct(torch.from_numpy(b).cuda(), 7)
        x1, k1 = ctx.apply_direct(torch.from_numpy(b1).cuda(), 1)
    x = x.cpu().numpy()
    assert ku == 7 and k1 == 1
    assert float(np.abs(x[0]).max()) == 0.0
    assert _rel(x[1], O.direct_projection(A, b1, 7)) < 1e-10
    v = b1 / np.linalg.norm(b1)
    h = np.vdot(v, A @ v)
    ref1 = np.linalg.norm(b1) * np.sign(h.real) * v
    assert _rel(x1.cpu().numpy(), ref1) < 1e-12
