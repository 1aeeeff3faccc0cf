"""The device task list, executed on the host (no GPU).

`stc_plan_export_taskset` hands out the arrays the factorization kernel replays: tasks in
queue order, their updates (operand tiles, inner-dimension maps, row and column ranges),
the tiles with their stored columns and 16-column row extents.  This file runs that list
with numpy, one task after another in queue order (a topological order of the DAG), the
way the kernel does it: SYRK / GEMM products chunked by 16 inner columns and cut to the
chunk's row extents, the TRSM of a row slice by 32-column panels cut to the panel's row
extents, a row slice of a diagonal tile factored against the rows of the slices before
it.  It checks that

* the result equals the oracle's factor on every structural entry of L (so the update
  lists are complete and the inner-dimension maps pair the right columns), and
* every row or column the extents let the kernel skip is exactly zero in the operand
  (so skipping is exact, reading 13), and
* the completion word of every diagonal tile (its nfinal) holds exactly the (column
  group, row slice) bits its tasks set, groups outside a slice's band skipped.

Row slices 1, 2, 4 and 8 and both queue orders are covered.
"""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import build as B
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

KC = 16      # inner chunk of the tile products
PANEL = 32   # TRSM panel width
DIAG, OFF, SYRK, FWD, FILL = 0, 1, 2, 3, 4
DG, DSL = 16, 4   # column group width and slices per word of a diagonal tile's completion bits
T_OFF, T_DENSE, T_BAND = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    if B.stale():
        B.build()
    L.lib()


class Replay:
    def __init__(self, P, slices, bl, fwd=False):
        ex = lambda w: L.stc_plan_export_taskset(P.h, slices, int(bl) | (2 if fwd else 0), w)
        self.nb = P.info["nb"]
        self.tasks = ex(L.STC_TASKSET_TASKS).reshape(-1, 13)
        self.upds = ex(L.STC_TASKSET_UPDS).reshape(-1, 10)
        self.imap = ex(L.STC_TASKSET_IMAP).reshape(-1, 2)
        self.tiles = ex(L.STC_TASKSET_TILES).reshape(-1, 13)
        self.saind = ex(L.STC_TASKSET_SAIND)
        self.cext = ex(L.STC_TASKSET_CEXT).reshape(-1, 2)
        self.csc_map = ex(L.STC_TASKSET_CSC_MAP)
        self.pad = ex(L.STC_TASKSET_PAD_DIAG)
        self.value_map = P.export("value_map")
        self.perm = P.export("perm")
        self.fdoubles = P.factor_bytes(1) // 8
        self.skipped_checks = 0

    # ---- storage
    def off_view(self, F, t):
        off, sw = self.tiles[t, 0], self.tiles[t, 4]
        return F[off:off + self.nb * sw].reshape(sw, self.nb).T  # [row, stored column]

    def diag_full(self, F, t):
        nb = self.nb
        off, kind, kd = self.tiles[t, 0], self.tiles[t, 3], self.tiles[t, 7]
        if kind == T_DENSE:
            return np.tril(F[off:off + nb * nb].reshape(nb, nb).T)
        D = np.zeros((nb, nb))
        for r in range(nb):
            for c in range(max(0, r - kd), r + 1):
                D[r, c] = F[off + (kd + c - r) + r * (kd + 1)]
        return D

    def diag_store(self, F, t, D, rows=None):
        nb = self.nb
        off, kind, kd = self.tiles[t, 0], self.tiles[t, 3], self.tiles[t, 7]
        rows = range(nb) if rows is None else rows
        for r in rows:
            for c in range(0, r + 1):
                if kind == T_DENSE:
                    F[off + r + c * nb] = D[r, c]
                elif r - c <= kd:
                    F[off + (kd + c - r) + r * (kd + 1)] = D[r, c]
                else:
                    assert D[r, c] == 0.0, "fill outside the band of a diagonal tile"

    def logical(self, t, s):
        c0, aoff = self.tiles[t, 5], self.tiles[t, 6]
        s = np.asarray(s)
        return c0 + s if c0 >= 0 else self.saind[aoff + s]

    def ext(self, t, s0, s1):
        xoff = self.tiles[t, 12]
        if xoff < 0:
            return 0, self.nb
        q = np.arange(s0 // 16, s1 // 16 + 1)
        return int(self.cext[xoff + q, 0].min()), int(self.cext[xoff + q, 1].max())

    def inner(self, u, k0, K, b):
        _, _, kmap, _, ka0, kb0 = u[:6]
        if kmap < 0:
            return np.arange(k0, k0 + K) + (kb0 if b else ka0)
        return self.imap[kmap + k0:kmap + k0 + K, 1 if b else 0]

    def assert_zero_outside(self, M, lo, hi, what):
        assert np.all(M[:lo] == 0.0) and np.all(M[hi:] == 0.0), what
        self.skipped_checks += 1

    # ---- tasks
    def potrf(self, F, t):
        nb, sw = self.nb, self.tiles[t, 4]
        D = self.diag_full(F, t)
        S = D[:sw, :sw]
        Lw = np.linalg.cholesky(S + np.tril(S, -1).T)
        D[:sw, :sw] = Lw
        self.diag_store(F, t, D)

    def syrk_into(self, F, D, u, r0, d0, rb):
        A = self.off_view(F, u[0])
        for k0 in range(0, u[3], KC):
            K = min(KC, u[3] - k0)
            idx = self.inner(u, k0, K, False)
            lo, hi = self.ext(u[0], idx[0], idx[-1])
            self.assert_zero_outside(A[:, idx], lo, hi, "SYRK operand outside its extent")
            q0, e0, e1 = max(r0, lo), max(d0, lo), min(rb, hi)
            if e0 >= e1:
                continue
            U = A[e0:e1, idx] @ A[q0:e1, idx].T
            D[e0:e1, q0:e1] -= np.tril(U, e0 - q0)  # lower part only (column <= row)

    def off_task(self, F, tk):
        kind, o, dk, ub, ue, rs0, rs1, tr0, tr1 = tk[:9]
        nb = self.nb
        Ot = self.off_view(F, o)
        sw = self.tiles[o, 4]
        X = Ot[rs0:rs1].copy()
        oc0 = self.tiles[o, 5]
        for u in self.upds[ub:ue]:
            A, Bt = self.off_view(F, u[0]), self.off_view(F, u[1])
            for k0 in range(0, u[3], KC):
                K = min(KC, u[3] - k0)
                ia, ib = self.inner(u, k0, K, False), self.inner(u, k0, K, True)
                alo, ahi = self.ext(u[0], ia[0], ia[-1])
                blo, bhi = self.ext(u[1], ib[0], ib[-1])
                self.assert_zero_outside(A[:, ia], alo, ahi, "GEMM A outside its extent")
                self.assert_zero_outside(Bt[:, ib], blo, bhi, "GEMM B outside its extent")
                e0, e1 = max(u[6], alo), min(u[7], ahi)
                c0, c1 = u[8], u[9]
                if oc0 >= 0:
                    c0, c1 = max(c0, blo - oc0), min(c1, bhi - oc0)
                if e0 >= e1 or c0 >= c1:
                    continue
                rows_b = self.logical(o, np.arange(c0, c1))
                X[e0 - rs0:e1 - rs0, c0:c1] -= A[e0:e1, ia] @ Bt[np.ix_(rows_b, ib)].T
        # TRSM against L_kk restricted to the stored columns, by panels
        Lk = self.diag_full(F, dk)
        lc = self.logical(o, np.arange(sw))
        Ls = Lk[np.ix_(lc, lc)]
        for p in range(0, sw, PANEL):
            pw = min(PANEL, sw - p)
            lo, hi = self.ext(o, p, p + pw - 1)
            y0, y1 = max(tr0, lo), min(tr1, hi)
            panel = X[:, p:p + pw]
            keep = np.zeros(rs1 - rs0, dtype=bool)
            keep[max(y0 - rs0, 0):max(y1 - rs0, 0)] = True
            assert np.all(panel[~keep] == 0.0), "TRSM rows outside the panel's extent are not zero"
            if y0 < y1:
                Lpp = Ls[p:p + pw, p:p + pw]
                X[y0 - rs0:y1 - rs0, p:p + pw] = np.linalg.solve(Lpp, X[y0 - rs0:y1 - rs0, p:p + pw].T).T
            pn = p + pw
            if pn >= sw or y0 >= y1:
                continue
            for k0 in range(p, pn, KC):
                K = min(KC, pn - k0)
                lo, hi = self.ext(o, k0, k0 + K - 1)
                x0, x1 = max(tr0, lo), min(tr1, hi)
                if x0 < x1:
                    X[x0 - rs0:x1 - rs0, pn:] -= X[x0 - rs0:x1 - rs0, k0:k0 + K] @ Ls[pn:, k0:k0 + K].T
        Ot[rs0:rs1] = X

    def fwd_task(self, F, tk, bp, Y):
        # y_k = L_kk^{-1} (b_k - sum_n L_kn y_n) with the tiles as they stand at this point
        # of the queue (a tile that is not final yet gives a wrong y)
        t, nb = tk[1], self.nb
        k = self.tiles[t, 2]
        v = bp[k * nb:(k + 1) * nb].copy()
        for o in np.nonzero((self.tiles[:, 3] == T_OFF) & (self.tiles[:, 1] == k))[0]:
            lc = self.logical(o, np.arange(self.tiles[o, 4]))
            v -= self.off_view(F, o) @ Y[self.tiles[o, 2] * nb + lc]
        D = self.diag_full(F, t)
        sw = self.tiles[t, 4]
        Y[k * nb:k * nb + sw] = solve_triangular(D[:sw, :sw], v[:sw], lower=True)

    def col_range(self, k):
        # a block column's tiles are contiguous in the factor, up to the logdet partials
        nb = self.nb
        size = lambda t: nb * t[4] if t[3] == T_OFF else (nb * nb if t[3] == T_DENSE else (t[7] + 1) * nb)
        ends = {}
        for t in self.tiles:
            b, e = ends.get(t[2], (t[0], t[0]))
            ends[t[2]] = (min(b, t[0]), max(e, t[0] + size(t)))
        return ends[k]

    def fill_col(self, F, k, values):
        b, e = self.col_range(k)
        F[b:e] = 0.0
        m = (self.value_map >= b) & (self.value_map < e)
        F[self.value_map[m]] = values[m]
        p = self.pad[(self.pad >= b) & (self.pad < e)]
        F[p] = 1.0

    def run(self, values, rhs=None):
        self.dbits = {}
        nb, n = self.nb, len(self.perm)
        nt = (n + nb - 1) // nb
        bp = np.zeros(nt * nb)
        if rhs is not None:
            bp[:n] = rhs[self.perm]
        self.y = np.zeros(nt * nb)
        for t in range(len(self.tiles)):
            if self.tiles[t, 3] != T_OFF:
                self.dbits[t] = 0
        inside = bool((self.tasks[:, 0] == FILL).any() or (self.tasks[:, 12] > 0).any())
        if inside:
            # the values arrive column by column inside the launch: anything a task reads
            # before its column is filled is NaN and shows in the result
            F = np.full(self.fdoubles, np.nan)
        else:
            F = np.zeros(self.fdoubles)
            F[self.value_map] = values
            F[self.pad] = 1.0
        nb = self.nb
        for tk in self.tasks:
            kind, t = tk[0], tk[1]
            if tk[12] > 0:  # a hosted value upload of a later block column, run first
                assert kind == SYRK and tk[10] == 1
                self.fill_col(F, tk[12] - 1, values)
            if kind == FILL:
                self.fill_col(F, self.tiles[t, 2], values)
                continue
            if tk[9] > 0:   # a hosted forward-substitution step, run first
                assert kind == DIAG or (kind == SYRK and tk[10] == 0)
                self.fwd_task(F, (FWD, tk[9] - 1), bp, self.y)
            if kind == DIAG:
                for g in range((self.tiles[t, 4] + DG - 1) // DG):
                    self.dbits[t] |= 1 << (g * DSL)
                D = self.diag_full(F, t)
                for u in self.upds[tk[3]:tk[4]]:
                    self.syrk_into(F, D, u, u[8], u[6], u[7])
                self.diag_store(F, t, D)
                self.potrf(F, t)
            elif kind == SYRK:
                rs0, rs1, sl = tk[5], tk[6], tk[10]
                assert rs0 % DG == 0 and rs1 - rs0 <= 64 and sl < DSL
                D = self.diag_full(F, t)
                for u in self.upds[tk[3]:tk[4]]:
                    assert rs0 <= u[6] and u[7] <= rs1
                    self.syrk_into(F, D, u, u[8], u[6], u[7])
                # the rows' factorization: columns [0, rs0) against the earlier slices' rows
                # (final: they come earlier in the queue), then the own diagonal block
                kd = self.tiles[t, 7]
                if rs0 > 0:
                    X = solve_triangular(D[:rs0, :rs0], D[rs0:rs1, :rs0].T, lower=True).T
                    for g0 in range(0, rs0, DG):
                        if g0 + DG <= rs0 - kd:   # skipped by the kernel: zero in these rows
                            assert np.all(X[:, g0:g0 + DG] == 0.0), "skipped group not zero"
                            self.skipped_checks += 1
                        else:
                            self.dbits[t] |= 1 << ((g0 // DG) * DSL + sl)
                    D[rs0:rs1, :rs0] = X
                    S = D[rs0:rs1, rs0:rs1] - X @ X.T
                else:
                    S = D[rs0:rs1, rs0:rs1]
                S = np.tril(S)
                D[rs0:rs1, rs0:rs1] = np.linalg.cholesky(S + np.tril(S, -1).T)
                for g in range(rs0 // DG, (rs1 + DG - 1) // DG):
                    self.dbits[t] |= 1 << (g * DSL + sl)
                self.diag_store(F, t, D, rows=range(rs0, rs1))
            elif kind == FWD:
                self.fwd_task(F, tk, bp, self.y)
            else:
                self.off_task(F, tk)
        for t, bits in self.dbits.items():
            assert bits == (self.tiles[t, 10] & 0xffffffff), "completion bits of diagonal tile %d" % t
        return F[self.csc_map]


def _cases():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(16, 16, 2)
    yield "bordered_nd_nb16", Ap, Ai, Ax, dict(coords=coords, nb=16, route="semisparse", nd_leaf=16)
    yield "bordered_nd_dense_nb32", Ap, Ai, Ax, dict(coords=coords, nb=32, route="dense", nd_leaf=16)
    Ap, Ai, Ax = I.band(700, 40, 1)
    yield "band_nb32", Ap, Ai, Ax, dict(nb=32, ordering="natural", route="semisparse")
    yield "band_nb128", Ap, Ai, Ax, dict(nb=128, ordering="natural", route="semisparse")
    Ap, Ai, coords = I.stcov_pattern(7, 6, 5, 3)
    Ax = I.stcov_values((2.0, 0.7, 0.5), 7, 6, 5, 3)
    yield "stcov_nd_nb16", Ap, Ai, Ax, dict(coords=coords, nb=16, nd_leaf=20, route="semisparse")
    Ap, Ai, Ax = I.random_spd(400, 0.008, 5)
    yield "random_rcm_nb8", Ap, Ai, Ax, dict(nb=8, ordering="rcm", route="semisparse")
    yield "random_rcm_nb24", Ap, Ai, Ax, dict(nb=24, ordering="rcm", route="semisparse")
    Ap, Ai, Ax, coords = I.fem3d(7, 6, 6)
    yield "fem_dense_nb16", Ap, Ai, Ax, dict(coords=coords, nb=16, route="dense", nd_leaf=20)


CASES = list(_cases())


@pytest.mark.parametrize("slices,bl", [(1, False), (2, False), (4, False), (8, False), (2, True)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_device_task_list_reproduces_oracle(case, slices, bl):
    name, Ap, Ai, Ax, kw = case
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, **kw)
    R = Replay(P, slices, bl)
    got = R.run(Ax)
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lo, info = F.factor(Ax)
    assert info == 0
    col = np.repeat(np.arange(n), np.diff(F.Lp))
    scale = np.maximum.reduceat(np.abs(Lo), F.Lp[:-1])[col]
    assert np.max(np.abs(got - Lo) / scale) <= 1e-12, name
    assert R.skipped_checks > 0


@pytest.mark.parametrize("slices,bl", [(2, False), (4, False), (8, True)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_forward_substitution_tasks(case, slices, bl):
    # the task set of the fused factorization + solve: its factor is the plain set's, and
    # each forward-substitution task, executed where it sits in the queue, gives
    # y = L^{-1} P b (so every tile it reads is final there)
    from scipy.sparse.linalg import spsolve_triangular
    import scipy.sparse as sp
    name, Ap, Ai, Ax, kw = case
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, **kw)
    b = np.random.default_rng(3).standard_normal(n)
    R = Replay(P, slices, bl, fwd=True)
    # every block's forward step exactly once: hosted by a waiting diagonal task or its own
    hosted = R.tiles[R.tasks[R.tasks[:, 9] > 0, 9] - 1, 2]
    own = R.tiles[R.tasks[R.tasks[:, 0] == FWD, 1], 2]
    assert sorted(np.concatenate([hosted, own])) == list(range((n + P.info["nb"] - 1) // P.info["nb"]))
    if name in ("band_nb128", "band_nb32") or (name == "bordered_nd_nb16" and not bl):
        assert len(hosted) > 0, "no forward step hosted"
    if name == "band_nb128":
        assert (R.tasks[:, 12] > 0).sum() >= len(hosted) // 2, "value upload not hosted"
    got = R.run(Ax, b)
    assert not np.isnan(got).any()
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lo, info = F.factor(Ax)
    assert np.array_equal(got, Replay(P, slices, bl).run(Ax))
    Lm = sp.csr_matrix(sp.csc_matrix((Lo, F.Li, F.Lp), shape=(n, n)))
    y = spsolve_triangular(Lm, b[F.perm], lower=True)
    assert np.max(np.abs(R.y[:n] - y)) <= 1e-12 * np.max(np.abs(y)), name


def test_queue_order_is_topological():
    # every tile a task reads (update operands, the diagonal tile of a TRSM) is complete,
    # i.e. all of its producing tasks come earlier in the queue (a row slice of a diagonal
    # tile after the slices before it)
    Ap, Ai, Ax, coords = I.laplace2d_bordered(16, 16, 2)
    P = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=16)
    for slices, bl in ((1, False), (2, False), (4, True), (8, False)):
        R = Replay(P, slices, bl)
        last = {}
        for i, tk in enumerate(R.tasks):
            last[tk[1]] = i
        for i, tk in enumerate(R.tasks):
            for u in R.upds[tk[3]:tk[4]]:
                assert last[u[0]] < i and last[u[1]] < i, (slices, bl, i)
            if tk[0] == OFF:
                assert last[tk[2]] < i
        # the row slices of a diagonal tile: in row order, contiguous, covering its width
        for t in {tk[1] for tk in R.tasks if tk[0] == SYRK}:
            rows = [(tk[5], tk[6], tk[10]) for tk in R.tasks if tk[0] == SYRK and tk[1] == t]
            assert [r[2] for r in rows] == list(range(len(rows)))
            assert rows[0][0] == 0 and rows[-1][1] == R.tiles[t, 4]
            assert all(rows[j][1] == rows[j + 1][0] for j in range(len(rows) - 1))


def _spd_from_pattern(n, rows, cols, seed):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    M = sp.coo_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, n)).tocsc()
    M = M + M.T
    M = M + sp.diags(np.asarray(abs(M).sum(axis=1)).ravel() + 1.0)
    return I.lower_csc(M)


EDGE = [
    ("n=1", 1, [], []),
    ("n=2", 2, [1], [0]),
    ("diagonal", 50, [], []),
    ("n=7 single ragged tile", 7, [3, 6, 5], [0, 2, 1]),
    ("dense", 40, *[list(x) for x in np.tril_indices(40, -1)]),
    ("n=64 tridiagonal (multiple of n_b)", 64, list(range(1, 64)), list(range(63))),
    ("disconnected blocks", 30, [1, 2, 20, 25], [0, 1, 18, 19]),
    ("one dense last row", 33, [32] * 32, list(range(32))),
]


@pytest.mark.parametrize("nb", [8, 32, 128])
@pytest.mark.parametrize("edge", EDGE, ids=lambda e: e[0])
def test_edge_patterns(edge, nb):
    # degenerate sizes and structures: both routes, two orderings, three slice counts
    name, n, r, c = edge
    Ap, Ai, Ax = _spd_from_pattern(n, np.array(r, dtype=int), np.array(c, dtype=int), 0)
    for route in ("semisparse", "dense"):
        for ordering in ("natural", "rcm"):
            P = Plan(n, Ap, Ai, nb=nb, route=route, ordering=ordering)
            F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
            Lo, info = F.factor(Ax)
            assert info == 0
            for slices, bl in ((1, False), (2, False), (8, True)):
                got = Replay(P, slices, bl).run(Ax)
                assert np.max(np.abs(got - Lo)) <= 1e-12 * np.max(np.abs(Lo)), (name, route, ordering, slices)


@pytest.mark.parametrize("seed", range(6))
def test_fused_task_sets_on_random_patterns(seed):
    # random patterns, tile sizes, orderings and slice counts: the fused task set executed
    # in queue order from a NaN factor (value uploads and forward steps where the queue
    # puts them) gives the oracle's factor and y = L^{-1} P b, so every task comes after
    # what it reads
    from scipy.sparse.linalg import spsolve_triangular
    import scipy.sparse as sp
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(150, 700))
    Ap, Ai, Ax = I.random_spd(n, float(rng.uniform(0.004, 0.03)), seed)
    nb = int(rng.choice([8, 16, 32, 64]))
    P = Plan(n, Ap, Ai, nb=nb, ordering=str(rng.choice(["rcm", "natural"])), route="semisparse")
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lo, info = F.factor(Ax)
    assert info == 0
    b = rng.standard_normal(n)
    Lm = sp.csr_matrix(sp.csc_matrix((Lo, F.Li, F.Lp), shape=(n, n)))
    y = spsolve_triangular(Lm, b[F.perm], lower=True)
    col = np.repeat(np.arange(n), np.diff(F.Lp))
    scale = np.maximum.reduceat(np.abs(Lo), F.Lp[:-1])[col]
    for slices, bl in ((1, False), (2, False), (4, True), (8, False)):
        R = Replay(P, slices, bl, fwd=True)
        got = R.run(Ax, b)
        assert not np.isnan(got).any()
        assert np.max(np.abs(got - Lo) / scale) <= 1e-12, (seed, slices, bl)
        assert np.max(np.abs(R.y[:n] - y)) <= 1e-11 * np.max(np.abs(y)), (seed, slices, bl)
