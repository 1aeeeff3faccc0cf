"""Pins for the CPU oracle: each check ties it to something other than itself.

Pins used (none of them re-types the oracle's own formula):
* numpy.linalg.cholesky / slogdet / solve / inv on dense copies (library routines);
* closed-form log-determinants (Dirichlet and Neumann Laplacian eigenvalues, AR1);
* the AR1 covariance rho^|i-j| / (1 - rho^2) for the selected inverse;
* brute-force dense boolean elimination for the symbolic factor;
* the paper's worked examples (Sec. 4.1 active columns, Sec. 4.3 banded tile);
* hand-derived task lists and ND orderings;
* a dense numpy tile executor driven by the oracle's Algorithm-1 task list, which must
  reproduce numpy's Cholesky (pins the order and completeness of the task list);
* central finite differences for gradients;
* exact rational arithmetic on small integer matrices (cofactor determinant, Cramer's rule);
* the block-determinant identity through the Schur complement of the border;
* closed-form theta derivatives of the border-free spatio-temporal log-determinant.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def full_sym(n, Ap, Ai, Ax):
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    return (A + sp.tril(A, -1).T).tocsc()


def dense_lower_pattern(n, Lp, Li):
    M = np.zeros((n, n), dtype=bool)
    for j in range(n):
        M[Li[Lp[j]:Lp[j + 1]], j] = True
    return M


# --------------------------------------------------------------------------- numeric
@pytest.mark.parametrize("n,density,seed", [(30, 0.1, 0), (60, 0.05, 1), (80, 0.3, 2)])
def test_cholesky_matches_numpy_dense(n, density, seed):
    Ap, Ai, Ax = I.random_spd(n, density, seed)
    perm = np.random.default_rng(seed).permutation(n)
    F = O.OracleFactor(n, Ap, Ai, perm)
    Lx, info = F.factor(Ax)
    assert info == 0
    A = full_sym(n, Ap, Ai, Ax).toarray()[np.ix_(perm, perm)]
    Lref = np.linalg.cholesky(A)
    L = O.to_dense_lower(n, F.Lp, F.Li, Lx)
    assert np.max(np.abs(L - Lref)) <= 1e-13 * np.max(np.abs(Lref))
    # every numerically non-zero entry of numpy's factor lies in the symbolic pattern
    pat = dense_lower_pattern(n, F.Lp, F.Li)
    assert not np.any((np.abs(Lref) > 1e-300) & ~pat)


def test_llt_invariant_config1():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, info = F.factor(Ax)
    assert info == 0
    L = sp.csc_matrix((Lx, F.Li, F.Lp), shape=(n, n))
    Ap_ = full_sym(n, Ap, Ai, Ax)[F.perm][:, F.perm]
    r = sp.linalg.norm(L @ L.T - Ap_) / sp.linalg.norm(Ap_)
    assert r <= 1e-14


def test_not_spd_reports_first_bad_column():
    # tridiagonal with a negative pivot appearing at column 3 (0-based)
    n = 6
    A = np.diag([4.0, 4.0, 4.0, -1.0, 4.0, 4.0]) + np.diag(np.full(n - 1, 1.0), -1) + np.diag(np.full(n - 1, 1.0), 1)
    Ap, Ai, Ax = I.lower_csc(sp.csc_matrix(A))
    F = O.OracleFactor(n, Ap, Ai)
    _, info = F.factor(Ax)
    assert info == 4
    # numpy agrees that the matrix is not SPD
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(A)


# --------------------------------------------------------------------------- logdet
def test_logdet_2d_dirichlet_closed_form():
    # 32x32 5-point Dirichlet Laplacian + 0.1 I, no border: eigenvalues
    # 4 - 2cos(a pi/33) - 2cos(b pi/33) + 0.1
    Ap, Ai, Ax, coords = I.laplace2d_bordered(32, 32, nborder=0)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, info = F.factor(Ax)
    a = np.arange(1, 33)
    lam = 4 - 2 * np.cos(a[:, None] * np.pi / 33) - 2 * np.cos(a[None, :] * np.pi / 33) + 0.1
    ref = np.sum(np.log(lam))
    assert abs(F.logdet(Lx) - ref) <= 1e-12 * abs(ref)


def test_logdet_config1_matches_numpy_slogdet():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, _ = F.factor(Ax)
    s, ref = np.linalg.slogdet(full_sym(n, Ap, Ai, Ax).toarray())
    assert s > 0 and abs(F.logdet(Lx) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("rho", [0.05, 0.5, 0.95])
def test_logdet_ar1_closed_form(rho):
    R = I.ar1_precision(50, rho)
    Ap, Ai, Ax = I.lower_csc(R)
    F = O.OracleFactor(50, Ap, Ai)
    Lx, _ = F.factor(Ax)
    assert abs(F.logdet(Lx) - np.log(1 - rho * rho)) <= 1e-12


def test_logdet_stcov_closed_form_small():
    # tau*R(rho) (x) S(kappa) on a 12 x 10 grid, 6 steps, no border:
    # n_f log tau + (nx ny) log(1-rho^2) + nt * [ny sum_a log(k2+mu_a) + nx sum_b log(k2+mu_b)]
    nx, ny, nt = 12, 10, 6
    tau, rho, kappa = 2.5, 0.7, 0.4
    Ap, Ai, coords = I.stcov_pattern(nx, ny, nt, 0)
    Ax = I.stcov_values((tau, rho, kappa), nx, ny, nt, 0)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, info = F.factor(Ax)
    assert info == 0
    k2 = kappa * kappa
    mux = 2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
    muy = 2 - 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
    ldS = ny * np.sum(np.log(k2 + mux)) + nx * np.sum(np.log(k2 + muy))
    ref = n * np.log(tau) + nx * ny * np.log(1 - rho * rho) + nt * ldS
    assert abs(F.logdet(Lx) - ref) <= 1e-11 * abs(ref)


def test_logdet_fem3d_unit_conductance_closed_form():
    # Neumann 7-point Laplacian on 8^3 + 1e-3 I: eigenvalues sum of (2-2cos(pi a/8)) + 1e-3
    m = 8
    Ap, Ai, Ax, coords = I.fem3d(m, m, m, unit_conductance=True)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, _ = F.factor(Ax)
    e = 2 - 2 * np.cos(np.pi * np.arange(m) / m)
    lam = e[:, None, None] + e[None, :, None] + e[None, None, :] + 1e-3
    ref = np.sum(np.log(lam))
    assert abs(F.logdet(Lx) - ref) <= 1e-10 * abs(ref)


def _det_cofactor(M):
    """Exact determinant of a small matrix of Fractions by Laplace expansion along row 0."""
    m = len(M)
    if m == 1:
        return M[0][0]
    tot = Fraction(0)
    for c in range(m):
        if M[0][c] != 0:
            minor = [row[:c] + row[c + 1:] for row in M[1:]]
            tot += (-1) ** c * M[0][c] * _det_cofactor(minor)
    return tot


@pytest.mark.parametrize("n,seed", [(3, 0), (5, 1), (7, 2), (8, 3)])
def test_logdet_and_solve_vs_exact_rational_arithmetic(n, seed):
    # integer SPD matrix (strictly diagonally dominant, random sparsity): the determinant by
    # cofactor expansion and the solution by Cramer's rule, both in exact rationals
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(i):
            if rng.uniform() < 0.6:
                A[i, j] = A[j, i] = int(rng.integers(-5, 6))
    A[np.arange(n), np.arange(n)] = np.abs(A).sum(axis=1) + rng.integers(1, 4, n)
    b = rng.integers(-9, 10, n)
    Ap, Ai, Ax = I.lower_csc(sp.csc_matrix(A.astype(float)))
    F = O.OracleFactor(n, Ap, Ai, rng.permutation(n))
    Lx, info = F.factor(Ax)
    assert info == 0
    Mq = [[Fraction(int(v)) for v in row] for row in A]
    det = _det_cofactor(Mq)
    assert det > 0
    assert abs(F.logdet(Lx) - math.log(det)) <= 1e-13 * max(1.0, math.log(det))
    x = F.solve(Lx, b.astype(float))
    for i in range(n):
        Mi = [row[:i] + [Fraction(int(b[r]))] + row[i + 1:] for r, row in enumerate(Mq)]
        xi = _det_cofactor(Mi) / det
        assert abs(x[i] - float(xi)) <= 1e-13 * max(1.0, abs(float(xi)))


def test_logdet_bordered_block_determinant():
    # logdet Q = logdet Q_ff + logdet(Q_bb - Q_bf Q_ff^-1 Q_fb): the field block is factored
    # on its own (border rows dropped), the 2x2 Schur complement is built from field solves
    # and its determinant taken by the 2x2 formula
    Ap, Ai, Ax, coords = I.laplace2d_bordered(20, 20, 2)
    n = len(Ap) - 1
    nf = n - 2
    Q = full_sym(n, Ap, Ai, Ax)
    Qff, Qfb, Qbb = Q[:nf, :nf], Q[:nf, nf:].toarray(), Q[nf:, nf:].toarray()
    Fa = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    full = Fa.logdet(Fa.factor(Ax)[0])
    fp, fi, fx = I.lower_csc(Qff)
    Ff = O.OracleFactor(nf, fp, fi, O.nd_lattice(coords[:nf]))
    Lf, info = Ff.factor(fx)
    assert info == 0
    Z = np.stack([Ff.solve(Lf, Qfb[:, k]) for k in range(2)], axis=1)
    S = Qbb - Qfb.T @ Z
    ref = Ff.logdet(Lf) + math.log(S[0, 0] * S[1, 1] - S[0, 1] * S[1, 0])
    assert abs(full - ref) <= 1e-12 * abs(ref)


# --------------------------------------------------------------------------- solve
def test_solve_matches_dense_and_residual():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(16, 16, 3)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, _ = F.factor(Ax)
    A = full_sym(n, Ap, Ai, Ax)
    b = I.rhs(n, 1)[0]
    x = F.solve(Lx, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1e-13
    xr = np.linalg.solve(A.toarray(), b)
    assert np.max(np.abs(x - xr)) <= 1e-12 * np.max(np.abs(xr))


# --------------------------------------------------------------------------- selinv
def test_selinv_matches_dense_inverse():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(12, 12, 2)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords))
    Lx, _ = F.factor(Ax)
    Sx = F.selinv(Lx)
    Ainv = np.linalg.inv(full_sym(n, Ap, Ai, Ax).toarray())[np.ix_(F.perm, F.perm)]
    col = np.repeat(np.arange(n), np.diff(F.Lp))
    ref = Ainv[F.Li, col]
    assert np.max(np.abs(Sx - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("rho", [0.3, 0.9])
def test_selinv_ar1_stationary_covariance(rho):
    # Sigma of the unit-innovation AR1 precision is rho^|i-j| / (1 - rho^2) everywhere
    nt = 40
    Ap, Ai, Ax = I.lower_csc(I.ar1_precision(nt, rho))
    F = O.OracleFactor(nt, Ap, Ai)
    Lx, _ = F.factor(Ax)
    Sx = F.selinv(Lx)
    col = np.repeat(np.arange(nt), np.diff(F.Lp))
    ref = rho ** np.abs(F.Li - col) / (1 - rho * rho)
    assert np.max(np.abs(Sx - ref)) <= 1e-12 * np.max(ref)


def test_grad_logdet_finite_differences_and_dense_inverse():
    Ap, Ai, Ax = I.random_spd(40, 0.1, 7)
    n = 40
    F = O.OracleFactor(n, Ap, Ai, np.random.default_rng(3).permutation(n))
    Lx, _ = F.factor(Ax)
    g = F.grad_logdet(F.selinv(Lx))
    Ainv = np.linalg.inv(full_sym(n, Ap, Ai, Ax).toarray())
    col = np.repeat(np.arange(n), np.diff(Ap))
    ref = np.where(Ai == col, 1.0, 2.0) * Ainv[Ai, col]
    assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))
    h = 1e-6
    for e in np.random.default_rng(0).choice(len(Ax), 8, replace=False):
        xp, xm = Ax.copy(), Ax.copy()
        xp[e] += h; xm[e] -= h
        fp = F.logdet(F.factor(xp)[0]); fm = F.logdet(F.factor(xm)[0])
        assert abs((fp - fm) / (2 * h) - g[e]) <= 1e-6 * max(1.0, abs(g[e]))


def test_theta_gradient_closed_form_without_border():
    # d logdet Q(theta)/d theta = sum_ij (d logdet/d a_ij)(d a_ij/d theta) on the lower
    # pattern; border-free closed forms: d/dtau = n/tau, d/drho = -nx ny 2 rho/(1-rho^2),
    # d/dkappa = nt [ny sum_a 2k/(k2+mu_a) + nx sum_b 2k/(k2+mu_b)]
    nx, ny, nt = 9, 7, 5
    Ap, Ai, coords = I.stcov_pattern(nx, ny, nt, 0)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords, 16))
    for tau, rho, kap in [(2.0, 0.6, 0.7), (0.3, 0.9, 1.5)]:
        th = (tau, rho, kap)
        Lx, info = F.factor(I.stcov_values(th, nx, ny, nt, 0))
        assert info == 0
        g = F.grad_logdet(F.selinv(Lx))
        got = I.stcov_dtheta(th, nx, ny, nt, 0) @ g
        mux = 2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
        muy = 2 - 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
        k2 = kap * kap
        ref = [n / tau, -nx * ny * 2 * rho / (1 - rho * rho),
               nt * (ny * np.sum(2 * kap / (k2 + mux)) + nx * np.sum(2 * kap / (k2 + muy)))]
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-10), (got, ref)


# --------------------------------------------------------------------------- symbolic
@pytest.mark.parametrize("n,density,seed", [(50, 0.05, 0), (120, 0.02, 1), (200, 0.01, 2)])
def test_symbolic_matches_bruteforce_elimination(n, density, seed):
    Ap, Ai, _ = I.random_spd(n, density, seed)
    perm = np.random.default_rng(seed + 10).permutation(n)
    F = O.OracleFactor(n, Ap, Ai, perm)
    A = full_sym(n, Ap, Ai, np.ones(len(Ai))).toarray()[np.ix_(perm, perm)] != 0
    M = np.tril(A)
    for k in range(n):  # dense boolean elimination
        r = np.nonzero(M[k + 1:, k])[0] + k + 1
        M[np.ix_(r, r)] |= np.tril(np.ones((len(r), len(r)), dtype=bool))
    M = np.tril(M)
    assert np.array_equal(dense_lower_pattern(n, F.Lp, F.Li), M)
    par = np.array([(np.nonzero(M[k + 1:, k])[0][0] + k + 1) if M[k + 1:, k].any() else -1 for k in range(n)])
    assert np.array_equal(F.parent, par)


def test_etree_tridiagonal_is_chain_and_arrowhead_has_no_fill():
    Ap, Ai, _ = I.tridiag(30, 0)
    F = O.OracleFactor(30, Ap, Ai)
    assert np.array_equal(F.parent, np.r_[np.arange(1, 30), -1])
    # arrowhead ordered border-last: no fill in the field; the (diagonal) border block
    # becomes a dense 3x3 lower triangle, i.e. exactly 3 fill entries
    Ap, Ai, _ = I.arrowhead(40, 3, 0)
    F = O.OracleFactor(40, Ap, Ai)
    assert F.nnzL == len(Ai) + 3


def test_nd_hand_derived_5x3_leaf3():
    # box x in [0,4], y in [0,2]: cut x=2; each half (2x3) cuts y=1 into 2-node leaves.
    # left  : (0,0),(1,0) | (0,2),(1,2) | sep (0,1),(1,1)  -> 0,1,10,11,5,6
    # right : 3,4 | 13,14 | 8,9 ; separator x=2: 2,7,12 ; then the border row 15
    coords = I.lattice_coords(5, 3, 1, nborder=1)
    perm = O.nd_lattice(coords, leaf_max=3)
    assert perm.tolist() == [0, 1, 10, 11, 5, 6, 3, 4, 13, 14, 8, 9, 2, 7, 12, 15]


def test_nd_is_permutation_and_separates():
    Ap, Ai, Ax, coords = I.fem3d(10, 9, 7)
    n = len(Ap) - 1
    perm = O.nd_lattice(coords)
    assert np.array_equal(np.sort(perm), np.arange(n))
    # top-level: the last separator plane splits the grid; no edge joins the two halves
    F = O.OracleFactor(n, Ap, Ai, perm)
    assert F.nnzL < n * (n + 1) // 2


# --------------------------------------------------------------------------- tiles
def test_paper_active_column_example():
    g = json.load(open(os.path.join(GOLD, "paper_active_column_tile.json")))
    nb = g["nb"]
    n = 2 * nb  # block column 0 decoupled internally, tile (1,0) holds the example
    A = np.eye(n) * 10.0
    for r, c in g["entries_row_col"]:
        A[nb + r, c] = A[c, nb + r] = 0.5
    Ap, Ai, Ax = I.lower_csc(sp.csc_matrix(A))
    F = O.OracleFactor(n, Ap, Ai)
    t = F.tile_map(nb)
    k = [i for i in range(len(t["I"])) if t["I"][i] == 1 and t["J"][i] == 0][0]
    a = t["aind"][t["aoff"][k]:t["aoff"][k] + t["nact"][k]]
    assert a.tolist() == g["aind"] and t["nact"][k] == g["nact"]
    assert bool(t["contig"][k]) == g["contiguous"] and bool(t["full"][k]) == g["full_width"]


def test_paper_banded_example_kd():
    g = json.load(open(os.path.join(GOLD, "paper_banded_diag_tile.json")))
    nb, kd = g["nb"], g["kd"]
    A = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            if abs(i - j) <= kd:
                A[i, j] = 4.0 if i == j else -0.5
    Ap, Ai, _ = I.lower_csc(sp.csc_matrix(A))
    t = O.OracleFactor(nb, Ap, Ai).tile_map(nb)
    assert t["kd"][0] == kd
    # the packed layout stores a_ij (i<=j) at (kd+i-j, j): check against the printed grid
    for i in range(nb):
        for j in range(i, min(nb, i + kd + 1)):
            assert g["packed"][kd + i - j][j] == "a%d%d" % (i, j)


@pytest.mark.parametrize("bw,nb", [(200, 128), (5, 8), (30, 16)])
def test_band_tiles_kd_and_active_columns(bw, nb):
    n = 40 * nb
    Ap, Ai = I.band_pattern(n, bw)
    t = O.OracleFactor(n, Ap, Ai).tile_map(nb)
    diag = t["I"] == t["J"]
    assert np.all(t["kd"][diag][:-1] == min(bw, nb - 1))
    if bw == 200:  # tile (k+2,k): active columns 56..127, contiguous, rows 0..71
        k = 5
        i = np.nonzero((t["I"] == k + 2) & (t["J"] == k))[0][0]
        a = t["aind"][t["aoff"][i]:t["aoff"][i] + t["nact"][i]]
        assert a.tolist() == list(range(56, 128)) and t["contig"][i] == 1 and t["full"][i] == 0
        assert (t["r0"][i], t["r1"][i]) == (0, 72)


def test_tile_map_matches_bruteforce():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(10, 10, 2)
    n = len(Ap) - 1
    F = O.OracleFactor(n, Ap, Ai, O.nd_lattice(coords, 8))
    nb = 16
    t = F.tile_map(nb)
    M = dense_lower_pattern(n, F.Lp, F.Li)
    nt = (n + nb - 1) // nb
    k = 0
    for J in range(nt):
        for Ib in range(J, nt):
            blk = M[Ib * nb:(Ib + 1) * nb, J * nb:(J + 1) * nb]
            cols = np.nonzero(blk.any(axis=0))[0]
            if len(cols) == 0:
                continue
            assert (t["I"][k], t["J"][k]) == (Ib, J)
            assert t["aind"][t["aoff"][k]:t["aoff"][k] + t["nact"][k]].tolist() == cols.tolist()
            rows = np.nonzero(blk.any(axis=1))[0]
            assert (t["r0"][k], t["r1"][k]) == (rows[0], rows[-1] + 1)
            if Ib == J:
                ii, jj = np.nonzero(blk)
                assert t["kd"][k] == np.max(ii - jj)
            k += 1
    assert k == len(t["I"])


def test_task_list_tridiagonal_hand_derived():
    # n=8, nb=2: tiles (k,k) and (k+1,k).  Per k: SYRK(k,k-1) if k>0, POTRF(k), TRSM(k+1,k).
    Ap, Ai, _ = I.tridiag(8, 0)
    t = O.OracleFactor(8, Ap, Ai).tile_map(2)
    exp = []
    for k in range(4):
        if k > 0:
            exp.append([2, -1, k, k - 1])
        exp.append([1, -1, k, -1])
        if k < 3:
            exp.append([3, k + 1, k, -1])
    assert t["tasks"].tolist() == exp


def _replay_dense(n, nb, A, tasks):
    """Dense numpy tile executor driven by an Algorithm-1 task list."""
    nt = (n + nb - 1) // nb
    N = nt * nb
    W = np.eye(N)
    W[:n, :n] = np.tril(A)
    blk = lambda i, j: W[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]
    for cs, m, k, nn in tasks:
        if cs == 2:
            blk(k, k)[:] -= np.tril(blk(k, nn) @ blk(k, nn).T)
        elif cs == 1:
            blk(k, k)[:] = np.linalg.cholesky(np.tril(blk(k, k)) + np.tril(blk(k, k), -1).T)
        elif cs == 4:
            blk(m, k)[:] -= blk(m, nn) @ blk(k, nn).T
        elif cs == 3:
            blk(m, k)[:] = np.linalg.solve(blk(k, k), blk(m, k).T).T
    return np.tril(W[:n, :n])


@pytest.mark.parametrize("case", ["c1small", "random", "band"])
def test_task_list_replay_reproduces_numpy_cholesky(case):
    if case == "c1small":
        Ap, Ai, Ax, coords = I.laplace2d_bordered(12, 12, 2)
        n = len(Ap) - 1
        perm = O.nd_lattice(coords, 16)
        nb = 16
    elif case == "random":
        n = 90
        Ap, Ai, Ax = I.random_spd(n, 0.03, 5)
        perm = np.random.default_rng(1).permutation(n)
        nb = 8
    else:
        n = 100
        Ap, Ai, Ax = I.band(n, 7, 3)
        perm = np.arange(n)
        nb = 6
    F = O.OracleFactor(n, Ap, Ai, perm)
    t = F.tile_map(nb)
    A = full_sym(n, Ap, Ai, Ax).toarray()[np.ix_(perm, perm)]
    L = _replay_dense(n, nb, A, t["tasks"])
    Lref = np.linalg.cholesky(A)
    assert np.max(np.abs(L - Lref)) <= 1e-12 * np.max(np.abs(Lref))


def test_features_and_selector():
    n = 40 * 16
    Ap, Ai = I.band_pattern(n, 20)
    F = O.OracleFactor(n, Ap, Ai)
    f = F.features(16)
    assert f["phi"] == 1.0 and f["sigma"] < 1.1
    assert O.select_route(**f) == O.ROUTE_SEMISPARSE
    # a dense matrix: every tile full -> dense route, phi = 1
    A = np.ones((64, 64)) + 64 * np.eye(64)
    Ap, Ai, _ = I.lower_csc(sp.csc_matrix(A))
    f = O.OracleFactor(64, Ap, Ai).features(16)
    assert f["rho"] == 1.0 and f["phi"] == 1.0
    assert O.select_route(**f) == O.ROUTE_DENSE
    assert O.select_route(phi=3.0, rho=0.5, sigma=1.0) == O.ROUTE_SUPERNODAL
    assert O.select_route(phi=1.5, rho=0.05, sigma=30.0) == O.ROUTE_SEMISPARSE
    assert O.select_route(phi=1.5, rho=0.05, sigma=3.0) == O.ROUTE_SUPERNODAL
