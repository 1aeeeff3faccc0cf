"""Python face of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference leg
may import this module.  The product path (paper_2609_29765_gb300) never does, and the
two share no code: the oracle is plain C (stc_oracle.c, compiled with gcc on first use)
plus the numpy below.

What it computes, with the paper's section for each step:

* ``OracleFactor(n, Ap, Ai, perm)`` -- permutation A_p = P A P^T, elimination tree and
  column structure of L (Sec. 3 symbolic factorization; Sec. 5.4 symbolic pipeline).
* ``.factor(Ax)``   -- left-looking column Cholesky, FP64 (exact factorization; Sec. 5.2
  at column granularity).
* ``.logdet / .solve`` -- 2 sum log L_jj; x = P^T L^-T L^-1 P b (Sec. 6.7).
* ``.selinv / .grad_logdet`` -- Takahashi selected inverse and d logdet/d a_ij
  = (2 - delta_ij) Sigma_ij (not in the paper: it leaves selected inversion to separate
  work, Sec. 6.2; textbook recurrence).
* ``.tile_map(nb) / .task_list(nb)`` -- Sec. 4 active-column tiles and Algorithm 1.
* ``features / select_route`` -- phi, rho, sigma and the selector of Sec. 5.1, with the
  precedence dense (rho>=0.90) > supernodal (phi>2.0) > semisparse (rho>=0.15 or
  sigma>=20) > supernodal.
* ``nd_lattice`` -- geometric nested dissection (this project's reading of Sec. 3's ND
  candidate: longest axis, midpoint plane, left/right/separator, leaves <= 64 nodes,
  lexicographic x-fastest, set-aside rows last).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build() -> str:
    """Compile the oracle's C code (gcc, -O2) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            build()
        L = C.CDLL(_SO)
        L.orc_nd_lattice.argtypes = [C.c_int64, _f64p, C.c_int64, _i64p]
        L.orc_nd_lattice.restype = C.c_int
        L.orc_permute_lower.argtypes = [C.c_int64, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p]
        L.orc_permute_lower.restype = C.c_int
        L.orc_symbolic.argtypes = [C.c_int64, _i64p, _i64p]
        L.orc_symbolic.restype = C.c_void_p
        L.orc_sym_nnz.argtypes = [C.c_void_p]
        L.orc_sym_nnz.restype = C.c_int64
        L.orc_sym_get.argtypes = [C.c_void_p, _i64p, _i64p, _i64p]
        L.orc_sym_get.restype = None
        L.orc_sym_free.argtypes = [C.c_void_p]
        L.orc_sym_free.restype = None
        L.orc_numeric.argtypes = [C.c_void_p, _i64p, _i64p, _f64p, _f64p]
        L.orc_numeric.restype = C.c_int64
        L.orc_logdet.argtypes = [C.c_void_p, _f64p]
        L.orc_logdet.restype = C.c_double
        L.orc_solve.argtypes = [C.c_void_p, _f64p, _i64p, _f64p, _f64p]
        L.orc_solve.restype = None
        L.orc_selinv.argtypes = [C.c_void_p, _f64p, _f64p]
        L.orc_selinv.restype = None
        L.orc_grad_logdet.argtypes = [C.c_void_p, _f64p, C.c_int64, _i64p, _i64p, _i64p, _f64p]
        L.orc_grad_logdet.restype = None
        L.orc_tile_map.argtypes = [C.c_void_p, C.c_int64]
        L.orc_tile_map.restype = C.c_void_p
        L.orc_tiles_sizes.argtypes = [C.c_void_p, _i64p]
        L.orc_tiles_sizes.restype = None
        L.orc_tiles_get.argtypes = [C.c_void_p, _i64p, _i64p]
        L.orc_tiles_get.restype = None
        L.orc_tiles_free.argtypes = [C.c_void_p]
        L.orc_tiles_free.restype = None
        L.orc_task_list.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_task_list.restype = C.c_int64
        _lib = L
        return L


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nd_lattice(coords: np.ndarray, leaf_max: int = 64) -> np.ndarray:
    """Geometric nested dissection on integral lattice coordinates ([n,3], NaN rows last)."""
    coords = _f64(coords)
    n = coords.shape[0]
    perm = np.empty(n, dtype=np.int64)
    if lib().orc_nd_lattice(n, coords.ravel(), leaf_max, perm) != 0:
        raise ValueError("nd_lattice: coordinates must be integral (or NaN for set-aside rows)")
    return perm


def permute_lower(n, Ap, Ai, perm):
    Ap, Ai, perm = _i64(Ap), _i64(Ai), _i64(perm)
    nnz = int(Ap[n])
    Bp = np.empty(n + 1, dtype=np.int64)
    Bi = np.empty(max(nnz, 1), dtype=np.int64)
    emap = np.empty(max(nnz, 1), dtype=np.int64)
    lib().orc_permute_lower(n, Ap, Ai, perm, Bp, Bi, emap)
    return Bp, Bi[:nnz], emap[:nnz]


class OracleFactor:
    """Symbolic analysis of one pattern under a fixed permutation (oracle side)."""

    def __init__(self, n: int, Ap, Ai, perm=None):
        self.n = int(n)
        self.Ap, self.Ai = _i64(Ap), _i64(Ai)
        self.perm = _i64(np.arange(n) if perm is None else perm)
        self.Bp, self.Bi, self.emap = permute_lower(self.n, self.Ap, self.Ai, self.perm)
        L = lib()
        self._h = L.orc_symbolic(self.n, self.Bp, self.Bi if self.Bi.size else np.zeros(1, np.int64))
        nnzl = L.orc_sym_nnz(self._h)
        self.parent = np.empty(self.n, dtype=np.int64)
        self.Lp = np.empty(self.n + 1, dtype=np.int64)
        self.Li = np.empty(max(nnzl, 1), dtype=np.int64)
        L.orc_sym_get(self._h, self.parent, self.Lp, self.Li)
        self.Li = self.Li[:nnzl]
        self.nnzL = int(nnzl)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_sym_free(h)
            self._h = None

    # -- numeric ---------------------------------------------------------
    def factor(self, Ax):
        """Left-looking Cholesky of A_p.  Returns (Lx, info); info = first bad column + 1."""
        Bx = np.zeros(self.Bi.shape[0])
        Bx[self.emap] = _f64(Ax)
        Lx = np.zeros(max(self.nnzL, 1))
        info = lib().orc_numeric(self._h, self.Bp, self.Bi, Bx, Lx)
        return Lx[: self.nnzL], int(info)

    def logdet(self, Lx) -> float:
        return float(lib().orc_logdet(self._h, _f64(Lx)))

    def solve(self, Lx, b):
        b = _f64(b)
        x = np.empty(self.n)
        lib().orc_solve(self._h, _f64(Lx), self.perm, b, x)
        return x

    def selinv(self, Lx):
        Sx = np.zeros(max(self.nnzL, 1))
        lib().orc_selinv(self._h, _f64(Lx), Sx)
        return Sx[: self.nnzL]

    def grad_logdet(self, Sx):
        g = np.empty(self.Ai.shape[0])
        lib().orc_grad_logdet(self._h, _f64(Sx), self.n, self.Ap, self.Ai, self.perm, g)
        return g

    # -- symbolic exports --------------------------------------------------
    def colcounts(self):
        return np.diff(self.Lp)

    def tile_map(self, nb: int) -> dict:
        L = lib()
        h = L.orc_tile_map(self._h, int(nb))
        sz = np.empty(3, dtype=np.int64)
        L.orc_tiles_sizes(h, sz)
        nt, ntiles, naind = (int(v) for v in sz)
        f = np.empty(max(ntiles, 1) * 9, dtype=np.int64)
        a = np.empty(max(naind, 1), dtype=np.int64)
        L.orc_tiles_get(h, f, a)
        ntask = L.orc_task_list(h, None)
        tasks = np.empty(max(ntask, 1) * 4, dtype=np.int64)
        L.orc_task_list(h, tasks.ctypes.data_as(C.c_void_p))
        L.orc_tiles_free(h)
        f = f[: ntiles * 9].reshape(ntiles, 9)
        return {
            "nb": int(nb), "nt": nt, "I": f[:, 0].copy(), "J": f[:, 1].copy(),
            "nact": f[:, 2].copy(), "aoff": f[:, 3].copy(), "contig": f[:, 4].copy(),
            "full": f[:, 5].copy(), "kd": f[:, 6].copy(), "r0": f[:, 7].copy(),
            "r1": f[:, 8].copy(), "aind": a[:naind].copy(),
            "tasks": tasks[: ntask * 4].reshape(ntask, 4).copy(),
        }

    def features(self, nb: int, tiles: dict | None = None) -> dict:
        """phi = nnz(L)/nnz(tril A); rho = mean |A|/n_b over active off-diagonal tiles;
        sigma = max column count of L / mean column count (Sec. 5.1)."""
        t = tiles if tiles is not None else self.tile_map(nb)
        off = t["I"] != t["J"]
        rho = float(np.mean(t["nact"][off] / nb)) if off.any() else 1.0
        cc = self.colcounts().astype(np.float64)
        return {"phi": self.nnzL / float(self.Ai.shape[0]), "rho": rho,
                "sigma": float(cc.max() / cc.mean()) if self.n else 0.0}


ROUTE_DENSE, ROUTE_SEMISPARSE, ROUTE_SUPERNODAL = 0, 1, 2


def select_route(phi: float, rho: float, sigma: float, rho_dense=0.90, phi_fill=2.0,
                 rho_semi=0.15, sigma_skew=20.0) -> int:
    """Selector of Sec. 5.1 with the default gates of Table 5."""
    if rho >= rho_dense:
        return ROUTE_DENSE
    if phi > phi_fill:
        return ROUTE_SUPERNODAL
    if rho >= rho_semi or sigma >= sigma_skew:
        return ROUTE_SEMISPARSE
    return ROUTE_SUPERNODAL


def to_dense_lower(n, Lp, Li, Lx) -> np.ndarray:
    """Dense n x n lower-triangular matrix from CSC arrays (small cases only)."""
    M = np.zeros((n, n))
    for j in range(n):
        for q in range(Lp[j], Lp[j + 1]):
            M[Li[q], j] = Lx[q]
    return M
