"""Seeded synthetic SPD inputs for the tile Cholesky (shared by tests, bench and oracle).

This module only *builds matrices*: sparsity patterns, values, lattice coordinates and
right-hand sides.  It holds none of the factorization's arithmetic, so both the CUDA
path and the CPU oracle may draw their inputs from it.

Every matrix is returned as the LOWER triangle (diagonal included) in CSC form with
rows sorted inside each column, in the original (unpermuted) order:

    Ap : int64[n+1]   column pointers
    Ai : int64[nnz]   row indices
    Ax : float64[nnz] values (or float64[batch, nnz] for a batch of value sets)

The workloads stand in for the paper's matrix classes (Sec. 2: banded SPDE fields,
spatio-temporal precisions with a dense covariate border, FEM operators); the paper's
60-matrix suite itself is not available, so each generator is a seeded synthetic
instance of one class:

* ``laplace2d_bordered`` -- 5-point Dirichlet Laplacian on an nx x ny grid + shift*I,
  with ``nborder`` dense border (arrowhead) rows, entries N(0, border_sd^2), each
  diagonal raised by the absolute row sums of the border couplings.
* ``band``               -- symmetric band, half-bandwidth ``bw``, off-diagonals
  U(-1,1) * 0.5/bw, diagonal 1 + absolute row sum.
* ``stcov``              -- tau * (AR1(rho) over nt steps (x) SPDE 9-point stencil
  (kappa^2 I + T)(x)(kappa^2 I + T) on an nx x ny grid) + dense border rows.
* ``fem3d``              -- 7-point graph Laplacian on an nx x ny x nz grid with
  lognormal(0,1) edge conductances + 1e-3 I (Neumann boundary).
* ``random_spd`` / ``arrowhead`` / ``tridiag`` -- small patterns for unit tests.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "lower_csc", "laplace2d_bordered", "band_pattern", "band_values", "band",
    "ar1_precision", "stcov_pattern", "stcov_values", "stcov_dtheta", "stcov_thetas",
    "fem3d", "random_spd", "arrowhead", "tridiag", "rhs", "lattice_coords",
]


def lower_csc(M: sp.spmatrix):
    """Lower triangle (with diagonal) of a symmetric sparse matrix as sorted CSC arrays."""
    L = sp.tril(sp.csc_matrix(M), format="csc")
    L.sum_duplicates()
    L.sort_indices()
    return (L.indptr.astype(np.int64), L.indices.astype(np.int64),
            L.data.astype(np.float64))


def lattice_coords(nx: int, ny: int, nz: int = 1, nborder: int = 0) -> np.ndarray:
    """[n,3] float64 lattice coordinates, node index x + nx*(y + ny*z); border rows NaN."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    if nborder:
        c = np.vstack([c, np.full((nborder, 3), np.nan)])
    return c


def _tridiag(m: int, diag: float, off: float) -> sp.csr_matrix:
    return sp.diags([np.full(m - 1, off), np.full(m, diag), np.full(m - 1, off)],
                    [-1, 0, 1], format="csr")


def _add_border(Qf: sp.spmatrix, nborder: int, sd: float, rng) -> sp.csr_matrix:
    """[[Qf + diag(|B| 1), B], [B^T, I + diag(1^T |B|)]] with B ~ N(0, sd^2)."""
    nf = Qf.shape[0]
    if nborder == 0:
        return sp.csr_matrix(Qf)
    B = rng.normal(0.0, sd, size=(nf, nborder))
    absB = np.abs(B)
    top = Qf + sp.diags(absB.sum(axis=1))
    bot = sp.diags(1.0 + absB.sum(axis=0))
    return sp.bmat([[top, sp.csr_matrix(B)], [sp.csr_matrix(B.T), bot]], format="csr")


def laplace2d_bordered(nx: int = 32, ny: int = 32, nborder: int = 2, shift: float = 0.1,
                       border_sd: float = 0.01, seed: int = 0):
    """5-point Dirichlet Laplacian (diag 4, -1 to neighbours) + shift*I, plus border rows.

    Returns (Ap, Ai, Ax, coords).  n = nx*ny + nborder.
    """
    rng = np.random.default_rng(seed)
    K = sp.kronsum(_tridiag(nx, 2.0, -1.0), _tridiag(ny, 2.0, -1.0), format="csr")
    Qf = K + shift * sp.identity(nx * ny, format="csr")
    Q = _add_border(Qf, nborder, border_sd, rng)
    Ap, Ai, Ax = lower_csc(Q)
    return Ap, Ai, Ax, lattice_coords(nx, ny, 1, nborder)


def band_pattern(n: int, bw: int):
    """Lower CSC pattern of a full band of half-bandwidth bw (rows j..min(j+bw, n-1))."""
    lens = np.minimum(bw, n - 1 - np.arange(n)) + 1
    Ap = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=Ap[1:])
    col = np.repeat(np.arange(n, dtype=np.int64), lens)
    Ai = col + (np.arange(Ap[-1], dtype=np.int64) - np.repeat(Ap[:-1], lens))
    return Ap, Ai


def band_values(n: int, bw: int, seed: int, Ap=None, Ai=None):
    """Values on band_pattern: off-diagonals U(-1,1)*0.5/bw, diagonal 1 + |row| sum."""
    if Ap is None:
        Ap, Ai = band_pattern(n, bw)
    rng = np.random.default_rng(seed)
    nnz = Ai.shape[0]
    col = np.repeat(np.arange(n, dtype=np.int64), np.diff(Ap))
    off = Ai != col
    Ax = np.empty(nnz, dtype=np.float64)
    Ax[off] = rng.uniform(-1.0, 1.0, size=int(off.sum())) * (0.5 / bw)
    a = np.abs(Ax[off])
    rs = np.bincount(Ai[off], weights=a, minlength=n) + np.bincount(col[off], weights=a, minlength=n)
    Ax[~off] = 1.0 + rs
    return Ax


def band(n: int = 200_000, bw: int = 200, seed: int = 0):
    Ap, Ai = band_pattern(n, bw)
    return Ap, Ai, band_values(n, bw, seed, Ap, Ai)


def ar1_precision(nt: int, rho: float) -> sp.csr_matrix:
    """Unit-innovation stationary AR1 precision: diag (1, 1+rho^2, ..., 1+rho^2, 1), off -rho."""
    d = np.full(nt, 1.0 + rho * rho)
    d[0] = d[-1] = 1.0
    return sp.diags([np.full(nt - 1, -rho), d, np.full(nt - 1, -rho)], [-1, 0, 1], format="csr")


def _spde(nx: int, ny: int, kappa: float) -> sp.csr_matrix:
    """(kappa^2 I + T_ny) (x) (kappa^2 I + T_nx), T = tridiag(-1,2,-1): a 9-point stencil."""
    Kx = _tridiag(nx, 2.0 + kappa * kappa, -1.0)
    Ky = _tridiag(ny, 2.0 + kappa * kappa, -1.0)
    return sp.kron(Ky, Kx, format="csr")


def _stcov_matrix(theta, nx, ny, nt, nborder, border_sd, border_seed):
    tau, rho, kappa = (float(v) for v in theta)
    Qf = tau * sp.kron(ar1_precision(nt, rho), _spde(nx, ny, kappa), format="csr")
    return _add_border(Qf, nborder, border_sd, np.random.default_rng(border_seed))


def stcov_pattern(nx: int = 60, ny: int = 60, nt: int = 50, nborder: int = 20):
    """Pattern (Ap, Ai) and lattice coordinates (x, y, t) of the spatio-temporal precision."""
    Ap, Ai, _ = lower_csc(_stcov_matrix((1.0, 0.5, 1.0), nx, ny, nt, nborder, 0.01, 0))
    return Ap, Ai, lattice_coords(nx, ny, nt, nborder)


def stcov_values(theta, nx: int = 60, ny: int = 60, nt: int = 50, nborder: int = 20,
                 border_sd: float = 0.01, border_seed: int = 0):
    """Values of Q(theta) = tau*(R(rho) (x) S(kappa)) + border on stcov_pattern's pattern."""
    _, _, Ax = lower_csc(_stcov_matrix(theta, nx, ny, nt, nborder, border_sd, border_seed))
    return Ax


def stcov_dtheta(theta, nx: int = 60, ny: int = 60, nt: int = 50, nborder: int = 20):
    """dQ/d(tau, rho, kappa) on stcov_pattern's lower CSC pattern, shape [3, nnz].

    The border block does not depend on theta.  Each derivative matrix is placed on the
    pattern by matching (column, row) keys, so pattern entries a derivative does not
    touch get 0.
    """
    tau, rho, kappa = (float(v) for v in theta)
    R = ar1_precision(nt, rho)
    S = _spde(nx, ny, kappa)
    dR = sp.diags([np.full(nt - 1, -1.0), np.r_[0.0, np.full(nt - 2, 2.0 * rho), 0.0],
                   np.full(nt - 1, -1.0)], [-1, 0, 1], format="csr")
    Kx = _tridiag(nx, 2.0 + kappa * kappa, -1.0)
    Ky = _tridiag(ny, 2.0 + kappa * kappa, -1.0)
    dS = 2.0 * kappa * (sp.kron(sp.identity(ny), Kx) + sp.kron(Ky, sp.identity(nx)))
    mats = [sp.kron(R, S), tau * sp.kron(dR, S), tau * sp.kron(R, dS)]
    Ap, Ai, _ = stcov_pattern(nx, ny, nt, nborder)
    n = len(Ap) - 1
    pkey = np.repeat(np.arange(n, dtype=np.int64), np.diff(Ap)) * n + Ai
    out = np.zeros((3, Ai.shape[0]))
    for k, M in enumerate(mats):
        Mp, Mi, Mx = lower_csc(M)
        mkey = np.repeat(np.arange(Mp.shape[0] - 1, dtype=np.int64), np.diff(Mp)) * n + Mi
        pos = np.searchsorted(pkey, mkey)
        if np.any(pos >= len(pkey)) or np.any(pkey[np.minimum(pos, len(pkey) - 1)] != mkey):
            raise AssertionError("derivative entry outside the pattern")
        out[k, pos] = Mx
    return out


def stcov_thetas(count: int, seed0: int = 0) -> np.ndarray:
    """theta_s = (tau, rho, kappa) log-uniform on [0.1,10] x [0.05,0.95] x [0.05,2], seed seed0+s."""
    lo = np.log([0.1, 0.05, 0.05])
    hi = np.log([10.0, 0.95, 2.0])
    out = np.empty((count, 3))
    for s in range(count):
        u = np.random.default_rng(seed0 + s).uniform(size=3)
        out[s] = np.exp(lo + u * (hi - lo))
    return out


def fem3d(nx: int = 64, ny: int = 64, nz: int = 64, seed: int = 0, shift: float = 1e-3,
          unit_conductance: bool = False):
    """7-point graph Laplacian with lognormal(0,1) edge conductances + shift*I.

    ``unit_conductance`` sets every c_e = 1 (the Neumann grid Laplacian).
    Returns (Ap, Ai, Ax, coords), node index x + nx*(y + ny*z).
    """
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols = [], []
    for a, b in ((idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]),
                 (idx[:-1, :, :], idx[1:, :, :])):
        rows.append(a.ravel()); cols.append(b.ravel())
    ei = np.concatenate(rows); ej = np.concatenate(cols)
    c = rng.lognormal(0.0, 1.0, size=ei.shape[0])
    if unit_conductance:
        c = np.ones_like(c)
    diag = np.bincount(ei, weights=c, minlength=n) + np.bincount(ej, weights=c, minlength=n) + shift
    M = sp.coo_matrix((np.r_[-c, -c, diag], (np.r_[ei, ej, np.arange(n)], np.r_[ej, ei, np.arange(n)])),
                      shape=(n, n))
    Ap, Ai, Ax = lower_csc(M)
    return Ap, Ai, Ax, lattice_coords(nx, ny, nz, 0)


def random_spd(n: int, density: float, seed: int, dominance: float = 1.0):
    """Random symmetric pattern, values U(-1,1), diagonal = dominance + |row| sum."""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, data_rvs=lambda k: rng.uniform(-1, 1, k))
    M = sp.tril(M, k=-1)
    M = M + M.T
    d = np.asarray(abs(M).sum(axis=1)).ravel() + dominance
    return lower_csc(M + sp.diags(d))


def arrowhead(n: int, nborder: int, seed: int):
    """Diagonal field with nborder dense trailing rows/columns (no fill)."""
    rng = np.random.default_rng(seed)
    Qf = sp.diags(1.0 + rng.uniform(size=n - nborder))
    return lower_csc(_add_border(Qf, nborder, 0.3, rng))


def tridiag(n: int, seed: int):
    rng = np.random.default_rng(seed)
    off = rng.uniform(-1, 1, size=n - 1)
    d = 2.5 + rng.uniform(size=n)
    return lower_csc(sp.diags([off, d, off], [-1, 0, 1]))


def rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand sides ~ N(0,1), shape [nrhs, n]."""
    return np.random.default_rng(seed).normal(size=(nrhs, n))
