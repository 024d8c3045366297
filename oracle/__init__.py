"""CPU oracle for sign(H_W(mu)) b by restarted LR-deflated multishift FOM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_0910_2927_gb300``) and never imports it.

Two layers, both FP64:

* O2, iterative (C, ``wilson.c`` / ``fomlr.c``): the Wilson kernel and
  Algorithm 1 (restarted FOM-LR(m,k)) in the A^2 reading of eq. (6.2).
* O1, dense (NumPy/SciPy, small lattices only): the dense matrix of H_W(mu),
  its eigendecomposition (critical eigenpairs for LR deflation, Sec. 4), the
  dense deflated rational target and the exact sign function; the direct
  projection of eq. (6.3) (non-restarted Arnoldi on A, sign(H_k) by Roberts'
  Newton iteration), the method the paper compares Algorithm 1 with.

Every function names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

_LIB = None


class _Lattice(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("antiperiodic", C.c_int * 4),
                ("mu", C.c_double), ("mass", C.c_double)]


class _Report(C.Structure):
    _fields_ = [("cycles", C.c_int), ("matvecs", C.c_int), ("converged", C.c_int),
                ("breakdown", C.c_int), ("res_est", C.c_double)]


def lib():
    """Load (building on first use) the C oracle."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_hw.argtypes = [C.POINTER(_Lattice), P, P, P]
        L.orc_hw.restype = None
        L.orc_hw_sites.argtypes = [C.POINTER(_Lattice), P, P, P, P, C.c_int64]
        L.orc_hw_sites.restype = None
        L.orc_kenney_laub.argtypes = [C.c_int, C.c_double, P, P]
        L.orc_kenney_laub.restype = C.c_int
        L.orc_fom_lr.argtypes = [C.POINTER(_Lattice), P, C.c_int, P, P, C.c_int, C.c_double,
                                 C.c_int, C.c_int, C.c_int, P, P, P, P, P, P,
                                 C.POINTER(_Report)]
        L.orc_fom_lr.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = C.c_int
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> int:
    """Threads of the oracle's later OpenMP regions; returns the count now in force."""
    return int(lib().orc_set_num_threads(int(n)))


def _lat(dims, mu, mass, antiperiodic):
    lt = _Lattice()
    for i in range(4):
        lt.dims[i] = int(dims[i])
        lt.antiperiodic[i] = int(antiperiodic[i])
    lt.mu = float(mu)
    lt.mass = float(mass)
    return lt


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- operator --

def hw(dims, links, psi, mu, mass=-1.6, antiperiodic=(0, 0, 0, 1)):
    """H_W(mu) psi = gamma5 D_W(mu) psi (Sec. 1; D_W(mu) as read in wilson.c)."""
    U = _c128(links)
    x = _c128(psi).reshape(-1)
    out = np.empty_like(x)
    lt = _lat(dims, mu, mass, antiperiodic)
    lib().orc_hw(C.byref(lt), _ptr(U), _ptr(x), _ptr(out))
    return out


def hw_sites(dims, links, psi, sites, mu, mass=-1.6, antiperiodic=(0, 0, 0, 1)):
    """H_W(mu) psi evaluated only at the listed sites; returns shape (len(sites), 12)."""
    U = _c128(links)
    x = _c128(psi).reshape(-1)
    out = np.zeros_like(x)
    st = np.ascontiguousarray(sites, dtype=np.int64)
    lt = _lat(dims, mu, mass, antiperiodic)
    lib().orc_hw_sites(C.byref(lt), _ptr(U), _ptr(x), _ptr(out), _ptr(st), st.size)
    return out.reshape(-1, 12)[st]


def dense_hw(dims, links, mu, mass=-1.6, antiperiodic=(0, 0, 0, 1)):
    """Dense n x n matrix of H_W(mu), column by column (small lattices only)."""
    n = 12 * int(np.prod(dims))
    A = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = hw(dims, links, e, mu, mass, antiperiodic)
        e[j] = 0.0
    return A


# ------------------------------------------------- rational approximation --

def kenney_laub(s, c=1.0):
    """Shifts and weights of eq. (6.2) with the scale c of Sec. 6 folded in.

    Returns (sigma', omega') with g_s(c t) = t sum omega'_i / (t^2 - sigma'_i).
    """
    sig = np.empty(s)
    om = np.empty(s)
    rc = lib().orc_kenney_laub(int(s), float(c), _ptr(sig), _ptr(om))
    if rc:
        raise ValueError("kenney_laub: need s >= 1 and c > 0")
    return sig, om


def kl_closed_form(t, s):
    """g_s(t) = ((t+1)^{2s} - (t-1)^{2s}) / ((t+1)^{2s} + (t-1)^{2s}), eq. (6.1)."""
    t = np.asarray(t, dtype=np.complex128)
    a = (t + 1) ** (2 * s)
    b = (t - 1) ** (2 * s)
    return (a - b) / (a + b)


def kl_partial_fractions(t, s, c=1.0):
    """g_s(c t) from the partial fractions of eq. (6.2)."""
    sig, om = kenney_laub(s, c)
    t = np.asarray(t, dtype=np.complex128)
    return t * sum(om[i] / (t * t - sig[i]) for i in range(s))


# ------------------------------------------------------------ Algorithm 1 --

def fom_lr(dims, links, b, mu, sigma, omega, k, tol, max_cycles=1000, project_each_cycle=True,
           R=None, L=None, lam=None, mass=-1.6, antiperiodic=(0, 0, 0, 1), want_shifts=False):
    """Restarted FOM-LR(m,k), Algorithm 1, in the A^2 reading of eq. (6.2).

    Returns (x, report, x_shift) where x approximates
    x_P + sum_i omega_i (A^2 - sigma_i)^{-1} A (I - P) b and x_shift[i] is the
    iterate of shifted system i (None unless want_shifts).
    """
    U = _c128(links)
    bb = _c128(b).reshape(-1)
    n = bb.size
    s = len(sigma)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    if R is None:
        m = 0
        Rc = Lc = lc = np.zeros(1, dtype=np.complex128)
    else:
        R = np.asarray(R)
        m = R.shape[1]
        Rc = _c128(R.T)      # column-major n x m == row-major m x n
        Lc = _c128(np.asarray(L).T)
        lc = _c128(lam)
    x = np.empty(n, dtype=np.complex128)
    xs = np.empty((s, n), dtype=np.complex128) if want_shifts else None
    rep = _Report()
    lt = _lat(dims, mu, mass, antiperiodic)
    rc = lib().orc_fom_lr(C.byref(lt), _ptr(U), s, _ptr(sig), _ptr(om), int(k), float(tol),
                          int(max_cycles), int(bool(project_each_cycle)), m, _ptr(Rc), _ptr(Lc),
                          _ptr(lc), _ptr(bb), _ptr(x), _ptr(xs) if xs is not None else None,
                          C.byref(rep))
    report = dict(status=rc, cycles=rep.cycles, matvecs=rep.matvecs, converged=bool(rep.converged),
                  breakdown=bool(rep.breakdown), res_est=rep.res_est)
    if rc not in (0, 3):
        raise RuntimeError(f"orc_fom_lr failed with status {rc}")
    return x, report, xs


# ------------------------------------------------------------ dense (O1) --

def eig(A):
    """Dense eigendecomposition A = X diag(w) X^{-1}; returns (w, X, X^{-1})."""
    w, X = np.linalg.eig(A)
    return w, X, np.linalg.inv(X)


def critical_eigenpairs(A, m, extra=0, decomposition=None):
    """LR deflation data of Sec. 4: the m eigenvalues of smallest |lambda|.

    Returns (R, L, lam, lam_next): right eigenvectors R (n x m), left
    eigenvectors L (n x m) normalised so that L^dag R = I (the rows of X^{-1}),
    the eigenvalues, and the next `extra` eigenvalues in the same order.
    Order: |lambda|, then Re lambda, then Im lambda.
    """
    w, X, Xinv = decomposition if decomposition is not None else eig(A)
    order = np.lexsort((w.imag, w.real, np.abs(w)))
    w = w[order]
    X = X[:, order]
    Xinv = Xinv[order, :]
    if m < len(w):
        gap = abs(w[m]) - abs(w[m - 1]) if m > 0 else 1.0
        if m > 0 and gap < 1e-8 * abs(w[m - 1]):
            raise ValueError("critical eigenvalue selection is ambiguous: |lambda_m| ~ |lambda_m+1|")
    R = X[:, :m].copy()
    L = Xinv[:m, :].conj().T.copy()
    return R, L, w[:m].copy(), w[m:m + extra].copy()


def deflated_target(A, b, sigma, omega, R=None, L=None, lam=None):
    """Dense x* = R sign(Re Lambda) L^dag b + sum_i omega_i (A^2 - sigma_i)^{-1} A (I - P) b.

    The split of eq. (4.2) with x_P from eq. (4.3) and the partial fractions of
    eq. (6.2) on the remainder; solved by dense LU, one solve per shift.
    """
    n = A.shape[0]
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    if R is None or R.shape[1] == 0:
        xP = np.zeros(n, dtype=np.complex128)
        r = b.copy()
    else:
        c = L.conj().T @ b
        xP = R @ (np.where(np.real(lam) > 0, 1.0, -1.0) * c)
        r = b - R @ c
    A2 = A @ A
    bt = A @ r
    x = xP.copy()
    eye = np.eye(n)
    for sg, om in zip(sigma, omega):
        x += om * np.linalg.solve(A2 - sg * eye, bt)
    return x


def gmres_lr(A, b, sigma, omega, k, tol, max_cycles=1000, R=None, L=None, lam=None, seed=None,
             want_shifts=False):
    """LR-deflated restarted multishift GMRES (GMRES-LR, Sec. 4 with Sec. 2's restarted multishift
    GMRES of the cited Frommer-Glassner work), A^2 reading of eq. (6.2), dense A, small cases.

    x = x_P + sum_i omega_i x_i with (A^2 - sigma_i) x_i = A (I - P) b.  One Krylov space of A^2
    per cycle, built by Arnoldi (CGS2) from the seed residual r.  The seed shift (default: the
    smallest |sigma_i|) takes the minimal-residual step, y_s = argmin ||beta e_1 - (Hbar_k -
    sigma_s I~) y||, leaving r <- V_{k+1} z, z = beta e_1 - (Hbar_k - sigma_s I~) y_s.  Every other
    shift keeps its residual collinear, r_i = rho_i r: (Hbar_k - sigma_i I~) y_i + rho_i' z =
    beta rho_i e_1, a square (k+1) x (k+1) system for (y_i, rho_i').  After each cycle the new
    seed residual is projected with I - P (eq. (4.5)).  Converged when every |rho_i| ||r|| <=
    tol ||A (I - P) b||.  Returns (x, cycles, [|rho_i| ||r|| / ||b~||])."""
    n = A.shape[0]
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    sigma = np.asarray(sigma, dtype=np.complex128)
    omega = np.asarray(omega, dtype=np.float64)
    s = len(sigma)
    seed = int(np.argmin(np.abs(sigma))) if seed is None else int(seed)
    if R is None or R.shape[1] == 0:
        xP = np.zeros(n, dtype=np.complex128)
        r0 = b.copy()
        proj = lambda v: v
    else:
        c = L.conj().T @ b
        xP = R @ (np.where(np.asarray(lam).real > 0, 1.0, -1.0) * c)
        r0 = b - R @ c
        proj = lambda v: v - R @ (L.conj().T @ v)
    bt = A @ r0
    bnorm = np.linalg.norm(bt)
    r = bt.copy()
    rho = np.ones(s, dtype=np.complex128)
    X = np.zeros((s, n), dtype=np.complex128)
    cycles = 0
    res = np.abs(rho) * np.linalg.norm(r) / bnorm
    while cycles < max_cycles and np.any(res > tol):
        beta = np.linalg.norm(r)
        V = np.zeros((n, k + 1), dtype=np.complex128)
        H = np.zeros((k + 1, k), dtype=np.complex128)
        V[:, 0] = r / beta
        kk = k
        for j in range(k):
            w = A @ (A @ V[:, j])
            for _ in range(2):
                h = V[:, :j + 1].conj().T @ w
                w = w - V[:, :j + 1] @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if abs(H[j + 1, j]) <= 1e-14 * np.linalg.norm(H[:j + 2, j]):
                kk = j + 1
                break
            V[:, j + 1] = w / H[j + 1, j]
        Hb = H[:kk + 1, :kk]
        It = np.eye(kk + 1, kk)
        e1 = np.zeros(kk + 1, dtype=np.complex128)
        e1[0] = beta
        # the seed's residual is the reference vector: rho[seed] = 1 throughout
        Ms = Hb - sigma[seed] * It
        ys = np.linalg.lstsq(Ms, e1, rcond=None)[0]
        z = e1 - Ms @ ys
        X[seed] += V[:, :kk] @ ys
        for i in range(s):
            if i == seed:
                continue
            Mi = np.concatenate([Hb - sigma[i] * It, z[:, None]], axis=1)
            sol = np.linalg.solve(Mi, rho[i] * e1)
            X[i] += V[:, :kk] @ sol[:kk]
            rho[i] = sol[kk]
        r = proj(V[:, :kk + 1] @ z)
        cycles += 1
        res = np.abs(rho) * np.linalg.norm(r) / bnorm
    if want_shifts:
        return xP + omega @ X, cycles, res, X
    return xP + omega @ X, cycles, res


def gamma5_diag(vol):
    """gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1) in the chiral basis of Sec. 1's
    H_W = gamma5 D_W, as the diagonal of the natural [site][spin][colour] layout."""
    return np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), vol)


def deflated_sign_matrix(A, sigma, omega, m=0, decomposition=None):
    """Dense F(A) = X f(Lambda) X^{-1} of the deflated rational sign function (eqs. (4.2)-(4.3)
    with (6.2)): f = sign(Re lambda) on the m critical eigenvalues (smallest |lambda|, the order
    of critical_eigenpairs) and f(t) = t sum_i omega_i / (t^2 - sigma_i) on the rest, so that
    F b = deflated_target(A, b, sigma, omega, R, L, lam) with those m pairs."""
    w, X, Xinv = decomposition if decomposition is not None else eig(A)
    order = np.lexsort((w.imag, w.real, np.abs(w)))
    w, X, Xinv = w[order], X[:, order], Xinv[order, :]
    sigma = np.asarray(sigma, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    f = w * np.sum(omega[None, :] / (w[:, None] ** 2 - sigma[None, :]), axis=1)
    f[:m] = np.where(w[:m].real > 0, 1.0, -1.0)
    return X @ (f[:, None] * Xinv)


def overlap_dense(F, vol):
    """The overlap operator D_ov = 1 + gamma5 F (Sec. 1: the operator the sign function is
    computed for), F a dense sign matrix (exact, or the deflated rational approximation)."""
    return np.eye(F.shape[0]) + gamma5_diag(vol)[:, None] * F


def dense_dhw_dmu(dims, links, mu, mass=-1.6, antiperiodic=(0, 0, 0, 1), h=1e-3):
    """Dense A' = dH_W/dmu.  H_W(mu) = H_0 + e^{mu} T_+ + e^{-mu} T_- (the chemical potential
    enters only the forward and backward time hops, Sec. 1), so
    H_W(mu + h) - H_W(mu - h) = 2 sinh(h) (e^{mu} T_+ - e^{-mu} T_-) = 2 sinh(h) A' exactly."""
    Hp = dense_hw(dims, links, mu + h, mass, antiperiodic)
    Hm = dense_hw(dims, links, mu - h, mass, antiperiodic)
    return (Hp - Hm) / (2.0 * math.sinh(h))


def rational_g(t, sigma, omega):
    """g(t) = t sum_i omega_i / (t^2 - sigma_i) (eq. (6.2) with the scale folded in) and g'(t)."""
    t = np.asarray(t)
    sigma = np.asarray(sigma, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    q = t[:, None] ** 2 - sigma[None, :]
    g = t * np.sum(omega[None, :] / q, axis=1)
    gp = np.sum(omega[None, :] * (-(t[:, None] ** 2) - sigma[None, :]) / q ** 2, axis=1)
    return g, gp


def frechet_dense(E, fvals, fprime, decomposition):
    """Frechet derivative of a matrix function of a diagonalisable A = X diag(w) X^{-1} along E
    (Daleckii-Krein): X (F ∘ (X^{-1} E X)) X^{-1}, F_jk the divided difference
    (f(w_j) - f(w_k)) / (w_j - w_k), and f'(w_j) on the diagonal and for equal eigenvalues."""
    w, X, Xinv = decomposition
    D = w[:, None] - w[None, :]
    same = np.abs(D) < 1e-12
    F = np.where(same, 0, (fvals[:, None] - fvals[None, :]) / np.where(same, 1, D))
    F[np.arange(len(w)), np.arange(len(w))] = fprime
    return X @ (F * (Xinv @ E @ X)) @ Xinv


def deflated_sign_derivative(A, E, sigma, omega, m=0, decomposition=None):
    """Derivative along E of the deflated rational sign function F(A) of deflated_sign_matrix:
    f = sign(Re lambda) on the m critical eigenvalues (derivative 0 there) and g elsewhere; the
    motion of the deflated eigenvectors enters through the divided differences between
    deflated and undeflated eigenvalues.  Returns (F, dF[E])."""
    w, X, Xinv = decomposition if decomposition is not None else eig(A)
    order = np.lexsort((w.imag, w.real, np.abs(w)))
    w, X, Xinv = w[order], X[:, order], Xinv[order, :]
    f, fp = rational_g(w, sigma, omega)
    f[:m] = np.where(w[:m].real > 0, 1.0, -1.0)
    fp[:m] = 0.0
    F = X @ (f[:, None] * Xinv)
    return F, frechet_dense(E, f, fp, (w, X, Xinv))


def sign_eig(A, decomposition=None):
    """Exact sign(A) = X sign(Re Lambda) X^{-1} (spectral definition, Sec. 1 footnote)."""
    w, X, Xinv = decomposition if decomposition is not None else eig(A)
    return (X * np.where(w.real > 0, 1.0, -1.0)) @ Xinv


def roberts_newton_sign(M, tol=1e-14, max_it=100):
    """sign(M) of a small dense matrix by Roberts' Newton iteration (Sec. 6, the
    direct-projection comparison): X_0 = M, X_{j+1} = (X_j + X_j^{-1}) / 2 until the
    update is below tol relative to X_j."""
    X = np.asarray(M, dtype=np.complex128).copy()
    for _ in range(max_it):
        Xn = 0.5 * (X + np.linalg.inv(X))
        if np.linalg.norm(Xn - X) <= tol * np.linalg.norm(Xn):
            return Xn
        X = Xn
    return X


def direct_projection(A, b, k, R=None, L=None, lam=None):
    """Direct projection of eq. (6.3): x = x_P + ||r|| V_k sign(H_k) e_1 with r = (I - P) b,
    x_P = R sign(Re Lambda) L^dag b, and V_k, H_k from k steps of Arnoldi on A started at r
    (classical Gram-Schmidt with one reorthogonalisation, eq. (2.4)); sign(H_k) by
    Roberts' Newton iteration.  For k = n (no breakdown) the result is sign(A) b exactly."""
    n = A.shape[0]
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    if R is None or R.shape[1] == 0:
        xP = np.zeros(n, dtype=np.complex128)
        r = b.copy()
    else:
        c = L.conj().T @ b
        xP = R @ (np.where(np.asarray(lam).real > 0, 1.0, -1.0) * c)
        r = b - R @ c
    beta = np.linalg.norm(r)
    V = np.zeros((n, k + 1), dtype=np.complex128)
    H = np.zeros((k + 1, k), dtype=np.complex128)
    V[:, 0] = r / beta
    kk = k
    for j in range(k):
        w = A @ V[:, j]
        for _ in range(2):
            h = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j].real <= 1e-14 * np.linalg.norm(H[:j + 2, j]):
            kk = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
    S = roberts_newton_sign(H[:kk, :kk])
    return xP + beta * (V[:, :kk] @ S[:, 0])


def sign_schur(A):
    """Exact sign(A) from the Schur form sorted right half-plane first.

    With A = Q T Q^dag, T = [[T11, T12], [0, T22]], spec(T11) in Re > 0 and
    spec(T22) in Re < 0: sign(T) = [[I, Z], [0, -I]] where T11 Z - Z T22 = 2 T12.
    """
    import scipy.linalg as sla
    T, Q, sdim = sla.schur(A.astype(np.complex128), output="complex", sort="rhp")
    n = A.shape[0]
    T11, T12, T22 = T[:sdim, :sdim], T[:sdim, sdim:], T[sdim:, sdim:]
    Z = sla.solve_sylvester(T11, -T22, 2 * T12)
    S = np.zeros((n, n), dtype=np.complex128)
    S[:sdim, :sdim] = np.eye(sdim)
    S[sdim:, sdim:] = -np.eye(n - sdim)
    S[:sdim, sdim:] = Z
    return Q @ S @ Q.conj().T


def rational_error_bound(lam_rest, s, c):
    """max over the non-deflated eigenvalues of |sign(c lambda) - g_s(c lambda)|.

    Closed form from eq. (6.1): for Re t > 0, g_s(t) = (1 - q^{2s}) / (1 + q^{2s})
    with q = (t - 1)/(t + 1), so sign(t) - g_s(t) = 2 q^{2s} / (1 + q^{2s});
    g_s is odd, which gives the Re t < 0 half.
    """
    t = c * np.asarray(lam_rest, dtype=np.complex128)
    t = np.where(t.real > 0, t, -t)
    q = (t - 1) / (t + 1)
    q2s = q ** (2 * s)
    return float(np.max(np.abs(2 * q2s / (1 + q2s)))) if t.size else 0.0


def scale_from_bounds(a_min, b_max):
    """c = ((m + r)(m - r))^{-1/2} of Sec. 6 for spectra in C(m,r) u C(-m,r).

    With the circle fitted to |lambda| in [a_min, b_max] on the real axis,
    m + r = b_max and m - r = a_min, so c = 1 / sqrt(a_min * b_max).
    """
    return 1.0 / math.sqrt(a_min * b_max)
