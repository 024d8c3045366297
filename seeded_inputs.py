"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the sign-function method itself: it only
draws gauge links, source vectors and test vectors from seeded generators.
Both the CPU oracle (``oracle/``) and the CUDA path consume what it returns;
neither side imports the other.

Recipe (stands in for the paper's unpublished lattice configurations, which
the paper uses in Sec. 6 for its 4^4 .. 10^4 experiments):

* gauge link U_nu(x) = exp(i * spread * sum_a g_a lambda_a / 2) with
  g_a ~ N(0, 1) and lambda_a the eight Gell-Mann matrices; exponentiated
  through the Hermitian eigendecomposition, then re-unitarised (Gram-Schmidt
  of rows 0 and 1, row 2 = conj(row0 x row1), so det U = 1);
* draw order: site lexicographic with x fastest, then direction x, y, z, t,
  then the 8 normals (one ``numpy.random.default_rng(seed)`` stream);
* Gaussian source b: (N(0,1) + i N(0,1)) / sqrt(2) per component;
* point sources: column 3*alpha + a is the unit vector at site 0, spin alpha,
  colour a.

Layouts (complex128, C order):
  links  [Lt][Lz][Ly][Lx][dir 4][3][3]   (row-major 3x3, dir = x, y, z, t)
  field  [Lt][Lz][Ly][Lx][spin 4][colour 3]
  block  [nrhs][site][spin][colour]  (nrhs independent fields back to back)
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann", "random_su3_links", "unit_links", "gaussian_field",
    "gaussian_block", "point_sources", "volume", "field_len", "random_gauge_transform",
    "CONFIG_SEEDS",
]

# Seeds per workload: gauge 1000+cfg, source 2000+cfg, cotangent 3000+cfg.
CONFIG_SEEDS = {cfg: (1000 + cfg, 2000 + cfg, 3000 + cfg) for cfg in range(1, 6)}


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def field_len(dims) -> int:
    """Complex components of one spinor field: 4 spins x 3 colours per site."""
    return 12 * volume(dims)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0][0, 1] = g[0][1, 0] = 1
    g[1][0, 1] = -1j
    g[1][1, 0] = 1j
    g[2][0, 0] = 1
    g[2][1, 1] = -1
    g[3][0, 2] = g[3][2, 0] = 1
    g[4][0, 2] = -1j
    g[4][2, 0] = 1j
    g[5][1, 2] = g[5][2, 1] = 1
    g[6][1, 2] = -1j
    g[6][2, 1] = 1j
    g[7][0, 0] = g[7][1, 1] = 1 / np.sqrt(3)
    g[7][2, 2] = -2 / np.sqrt(3)
    return g


def _reunitarise(u: np.ndarray) -> np.ndarray:
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3_links(dims, spread: float, seed: int, chunk: int = 1 << 16) -> np.ndarray:
    """Seeded random SU(3) links, shape (V, 4, 3, 3) complex128 (site x fastest)."""
    vol = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((vol, 4, 8))
    lam = gell_mann()
    out = np.empty((vol, 4, 3, 3), dtype=np.complex128)
    flat_g = g.reshape(-1, 8)
    flat_out = out.reshape(-1, 3, 3)
    for s in range(0, flat_g.shape[0], chunk):
        gg = flat_g[s:s + chunk]
        herm = 0.5 * spread * np.einsum("ka,aij->kij", gg, lam)
        w, q = np.linalg.eigh(herm)
        u = np.einsum("kij,kj,klj->kil", q, np.exp(1j * w), np.conj(q))
        flat_out[s:s + chunk] = _reunitarise(u)
    return out


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    out = np.zeros((volume(dims), 4, 3, 3), dtype=np.complex128)
    out[..., 0, 0] = out[..., 1, 1] = out[..., 2, 2] = 1
    return out


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site, shape (V, 3, 3)."""
    vol = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((vol, 8))
    herm = 0.5 * 2.0 * np.einsum("ka,aij->kij", g, gell_mann())
    w, q = np.linalg.eigh(herm)
    u = np.einsum("kij,kj,klj->kil", q, np.exp(1j * w), np.conj(q))
    return _reunitarise(u)


def gaussian_field(dims, seed: int) -> np.ndarray:
    """Complex Gaussian spinor field, shape (V*12,), unit variance per component."""
    rng = np.random.default_rng(seed)
    n = field_len(dims)
    z = rng.standard_normal((n, 2))
    return (z[:, 0] + 1j * z[:, 1]) / np.sqrt(2.0)


def gaussian_block(dims, nrhs: int, seed: int) -> np.ndarray:
    """nrhs independent complex Gaussian fields, shape (nrhs, V*12)."""
    rng = np.random.default_rng(seed)
    n = field_len(dims)
    z = rng.standard_normal((nrhs, n, 2))
    return (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)


def point_sources(dims, nrhs: int = 12) -> np.ndarray:
    """Spin-colour point sources at site 0: column 3*alpha + a, shape (nrhs, V*12)."""
    n = field_len(dims)
    out = np.zeros((nrhs, n), dtype=np.complex128)
    for c in range(nrhs):
        out[c, c % 12] = 1.0
    return out
