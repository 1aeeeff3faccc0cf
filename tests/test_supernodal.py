"""Host plan of the non-uniform supernodal tiling (Sec. 5.4), checked on the CPU.

* structure: the supernodes partition the columns, each panel's row list holds every
  structural entry of its columns, cells partition the rows below each diagonal block
  by owning supernode, panels do not overlap;
* relaxation: every supernode is a run of fundamental supernodes (computed here from
  their definition on the oracle's etree and column counts) or a 128-column panel of
  one, and every merge respects the stated amalgamation thresholds;
* numerics: a dense numpy executor that runs the exported task list on the exported
  cells (POTRF / TRSM / UPDATE with sorted-subset scatter) reproduces the oracle's L on
  every structural entry, leaves every explicit zero at 0.0 and gives the oracle's logdet.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import build as B
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

MAXW = 128


@pytest.fixture(scope="module", autouse=True)
def _built():
    if B.stale():
        B.build()
    L.lib()


def _dense_spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    return I.lower_csc(sp.csc_matrix(np.tril(A) + np.tril(A, -1).T))


def _cases():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(16, 16, 2)
    yield "laplace_bordered_nd", Ap, Ai, Ax, dict(coords=coords, ordering="nd", nd_leaf=16)
    Ap, Ai, coords = I.stcov_pattern(8, 7, 5, 3)
    Ax = I.stcov_values((1.5, 0.6, 0.8), 8, 7, 5, 3)
    yield "stcov_nd", Ap, Ai, Ax, dict(coords=coords, ordering="nd", nd_leaf=20)
    Ap, Ai, Ax, coords = I.fem3d(9, 8, 7)
    yield "fem3d_nd", Ap, Ai, Ax, dict(coords=coords, ordering="nd", nd_leaf=20)
    Ap, Ai, Ax = I.random_spd(300, 0.01, 4)
    yield "random_rcm", Ap, Ai, Ax, dict(ordering="rcm")
    Ap, Ai, Ax = I.band(900, 13, 2)
    yield "band_natural", Ap, Ai, Ax, dict(ordering="natural")
    Ap, Ai, Ax = I.arrowhead(400, 5, 1)
    yield "arrowhead_natural", Ap, Ai, Ax, dict(ordering="natural")
    Ap, Ai, Ax = _dense_spd(300, 3)
    yield "dense_300", Ap, Ai, Ax, dict(ordering="natural")


CASES = list(_cases())


def _plan(case):
    name, Ap, Ai, Ax, kw = case
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, nb=32, route="semisparse", **kw)
    return n, P


def _sn(P):
    nodes = P.export("sn_nodes")
    rows = P.export("sn_rows")
    rptr = np.concatenate([[0], np.cumsum(nodes[:, 2])])
    return nodes, rows, rptr, P.export("sn_cells"), P.export("sn_tasks")


def _fundamental(n, parent, Lp):
    cnt = np.diff(Lp)
    nchild = np.bincount(parent[parent >= 0], minlength=n)
    first = [j for j in range(n)
             if not (j > 0 and parent[j - 1] == j and cnt[j - 1] == cnt[j] + 1 and nchild[j] == 1)]
    return first + [n]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_supernodal_structure(case):
    n, P = _plan(case)
    nodes, rows, rptr, cells, _ = _sn(P)
    Lp, Li = P.export("Lp"), P.export("Li")
    first = nodes[:, 0]
    w = nodes[:, 1]
    assert first[0] == 0 and np.all(first[1:] == first[:-1] + w[:-1]) and first[-1] + w[-1] == n
    assert np.all((w >= 1) & (w <= MAXW))
    snof = np.repeat(np.arange(len(nodes)), w)
    end = 0
    for s, (f, ws, m, off) in enumerate(nodes):
        R = rows[rptr[s]:rptr[s + 1]]
        assert np.array_equal(R[:ws], np.arange(f, f + ws))
        assert np.all(np.diff(R) > 0)
        # the row list is the structure of the panel's last column below the diagonal
        last = f + ws - 1
        assert np.array_equal(R[ws:], Li[Lp[last] + 1:Lp[last + 1]])
        # every structural entry of the panel's columns is stored
        for j in range(f, f + ws):
            assert np.all(np.isin(Li[Lp[j]:Lp[j + 1]], R))
        assert off >= end and off % 4 == 0
        end = off + m * ws
        # cells: the diagonal block, then runs of rows by owning supernode, ascending
        C = cells[cells[:, 0] == s]
        assert tuple(C[0]) == (s, s, 0, ws)
        assert C[1:, 2].tolist() == ([ws] + C[1:-1, 3].tolist() if len(C) > 1 else [])
        if len(C) > 1:
            assert C[-1, 3] == m and np.all(np.diff(C[1:, 1]) > 0) and np.all(C[1:, 1] > s)
        for (_, J, r0, r1) in C[1:]:
            assert np.all(snof[R[r0:r1]] == J)


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_supernodal_relaxation_rule(case):
    n, P = _plan(case)
    nodes, _, _, _, _ = _sn(P)
    parent, Lp = P.export("etree"), P.export("Lp")
    cnt = np.diff(Lp)
    fund = _fundamental(n, parent, Lp)
    fset = set(fund)
    for f, ws, m, _ in nodes:
        e = f + ws
        inner = [b for b in fund if f < b < e]
        if f in fset and e in fset and not inner:
            continue  # one fundamental supernode (or all of one)
        if not inner:
            # a 128-column panel cut from one wide fundamental supernode
            lo = max(b for b in fund if b <= f)
            hi = min(b for b in fund if b >= e)
            assert hi - lo > MAXW and (f - lo) % MAXW == 0
            continue
        # a merged run of fundamental supernodes: explicit zeros within the thresholds
        assert f in fset and e in fset
        stored = ws * (ws + 1) / 2 + ws * (m - ws)
        z = (stored - cnt[f:e].sum()) / stored
        assert ws <= 4 or (ws <= 16 and z < 0.8) or (ws <= 48 and z < 0.1) or z < 0.05, (f, ws, z)


def test_supernodal_hand_derived():
    # tridiagonal, n = 10: column counts 2,...,2,1, fundamental supernodes {0},...,{7},
    # {8,9}; every merge keeps width <= 16 with explicit zeros below 80 % (at width 10:
    # 55 stored, 19 structural), so one supernode holds all ten columns
    Ap, Ai, _ = I.tridiag(10, 0)
    P = Plan(10, Ap, Ai, nb=8, ordering="natural")
    nodes, rows, _, cells, tasks = _sn(P)
    assert nodes.tolist() == [[0, 10, 10, 0]]
    assert tasks.tolist() == [[0, 0, -1, -1]]
    # dense n = 300: one fundamental supernode, cut into panels of 128, 128 and 44 columns
    Ap, Ai, _ = _dense_spd(300, 0)
    P = Plan(300, Ap, Ai, nb=32, ordering="natural")
    nodes, rows, _, cells, tasks = _sn(P)
    assert nodes[:, :3].tolist() == [[0, 128, 300], [128, 128, 172], [256, 44, 44]]
    assert cells.tolist() == [[0, 0, 0, 128], [0, 1, 128, 256], [0, 2, 256, 300],
                              [1, 1, 0, 128], [1, 2, 128, 172], [2, 2, 0, 44]]
    # left-looking: factor 0, TRSMs of its cells, then for 1: updates (1,1) and (2,1) from 0,
    # factor, TRSM; for 2: updates from 0 and 1, factor
    assert tasks.tolist() == [[0, 0, -1, -1], [1, 1, -1, -1], [1, 2, -1, -1],
                              [2, 3, 1, 1], [2, 4, 2, 1], [0, 3, -1, -1], [1, 4, -1, -1],
                              [2, 5, 2, 2], [2, 5, 4, 4], [0, 5, -1, -1]]


def _execute(n, P, Ap, Ai, Ax):
    """Run the exported supernodal task list with dense numpy kernels."""
    nodes, rows, rptr, cells, tasks = _sn(P)
    perm = P.export("perm")
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    arena = np.zeros(int(nodes[-1, 3] + nodes[-1, 1] * nodes[-1, 2]) + 4)
    M = [arena[off:off + m * ws].reshape(ws, m).T for (_, ws, m, off) in nodes]  # column-major views
    R = [rows[rptr[s]:rptr[s + 1]] for s in range(len(nodes))]
    snof = np.repeat(np.arange(len(nodes)), nodes[:, 1])
    col = np.repeat(np.arange(n), np.diff(Ap))
    a, b = iperm[Ai], iperm[col]
    i, j = np.maximum(a, b), np.minimum(a, b)
    for ii, jj, v in zip(i, j, Ax):
        s = snof[jj]
        M[s][np.searchsorted(R[s], ii), jj - nodes[s, 0]] = v
    for kind, c, x, y in tasks:
        J = cells[c, 0]
        if kind == 0:
            ws = nodes[J, 1]
            D = np.tril(M[J][:ws, :ws])
            M[J][:ws, :ws] = np.linalg.cholesky(D + np.tril(D, -1).T)
        elif kind == 1:
            ws = nodes[J, 1]
            r0, r1 = cells[c, 2:]
            Lkk = M[J][:ws, :ws]
            M[J][r0:r1] = np.linalg.solve(Lkk, M[J][r0:r1].T).T
        else:
            Isn, _, a0, a1 = cells[x]
            _, _, b0, b1 = cells[y]
            U = M[Isn][a0:a1] @ M[Isn][b0:b1].T
            tr = np.searchsorted(R[J], R[Isn][a0:a1])
            assert np.array_equal(R[J][tr], R[Isn][a0:a1]), "rows of (K,I) not a subset of J's rows"
            tc = R[Isn][b0:b1] - nodes[J, 0]
            assert np.all((tc >= 0) & (tc < nodes[J, 1]))
            t0, t1 = cells[c, 2:]
            assert np.all((tr >= t0) & (tr < t1)), "update lands outside its target cell"
            M[J][np.ix_(tr, tc)] -= U
    return nodes, R, M


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_supernodal_tasks_reproduce_oracle_factor(case):
    name, Ap, Ai, Ax, kw = case
    n, P = _plan(case)
    nodes, R, M = _execute(n, P, Ap, Ai, Ax)
    perm = P.export("perm")
    F = O.OracleFactor(n, Ap, Ai, perm)
    Lx, info = F.factor(Ax)
    assert info == 0
    scale = np.max(np.abs(Lx))
    snof = np.repeat(np.arange(len(nodes)), nodes[:, 1])
    covered = [np.zeros((len(R[s]), nodes[s, 1]), dtype=bool) for s in range(len(nodes))]
    for j in range(n):
        s = snof[j]
        rr = F.Li[F.Lp[j]:F.Lp[j + 1]]
        pos = np.searchsorted(R[s], rr)
        got = M[s][pos, j - nodes[s, 0]]
        assert np.max(np.abs(got - Lx[F.Lp[j]:F.Lp[j + 1]])) <= 1e-12 * scale, (name, j)
        covered[s][pos, j - nodes[s, 0]] = True
    for s in range(len(nodes)):
        ws = nodes[s, 1]
        lower = np.ones_like(covered[s])
        lower[:ws, :ws] = np.tril(np.ones((ws, ws), dtype=bool))
        assert np.all(M[s][lower & ~covered[s]] == 0.0), (name, s)  # explicit zeros stay zero
    ld = 2 * sum(np.sum(np.log(np.diag(M[s][:nodes[s, 1], :nodes[s, 1]]))) for s in range(len(nodes)))
    assert abs(ld - F.logdet(Lx)) <= 1e-12 * abs(F.logdet(Lx))


@pytest.mark.parametrize("seed", range(10))
def test_supernodal_random_patterns(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(20, 600))
    Ap, Ai, Ax = I.random_spd(n, float(rng.uniform(0.002, 0.08)), 40 + seed)
    kind = ["rcm", "natural", "given"][seed % 3]
    perm = rng.permutation(n) if kind == "given" else None
    P = Plan(n, Ap, Ai, nb=32, ordering=kind if perm is None else "auto", perm=perm)
    nodes, R, M = _execute(n, P, Ap, Ai, Ax)
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lx, info = F.factor(Ax)
    assert info == 0
    snof = np.repeat(np.arange(len(nodes)), nodes[:, 1])
    got = np.concatenate([M[snof[j]][np.searchsorted(R[snof[j]], F.Li[F.Lp[j]:F.Lp[j + 1]]), j - nodes[snof[j], 0]]
                          for j in range(n)])
    assert np.max(np.abs(got - Lx)) <= 1e-12 * np.max(np.abs(Lx))
    got2 = _execute_device_form(n, P, Ax)
    assert np.max(np.abs(got2 - Lx)) <= 1e-12 * np.max(np.abs(Lx))


def _execute_device_form(n, P, values):
    """Run the supernodal plan's device form with numpy, task by task in queue order,
    as a supernodal executor would: load the target rows, subtract every update through
    its row and column maps, then POTRF (diagonal cell) or TRSM (off-diagonal slice)."""
    cells = P.export("sn_dev_cells")
    tasks = P.export("sn_dev_tasks")
    upds = P.export("sn_dev_upds")
    maps = P.export("sn_dev_maps")
    nodes = P.export("sn_nodes")
    arena = np.zeros(int(nodes[-1, 3] + nodes[-1, 1] * nodes[-1, 2]) + 4)
    arena[P.export("sn_value_map")] = values

    def view(c):  # cell c as an h x w matrix view into the arena
        off, ld, h, w = cells[c, :4]
        return np.lib.stride_tricks.as_strided(arena[off:], shape=(h, w), strides=(8, 8 * ld))

    for kind, c, d, ub, ue, rs0, rs1, _ in tasks:
        X = view(c)[rs0:rs1].copy()
        for a, b, ar0, ar1, rmap, cmap, klen in upds[ub:ue]:
            assert cells[a, 3] == klen and cells[b, 3] == klen and cells[a, 4] == cells[b, 4]
            U = view(a)[ar0:ar1] @ view(b).T
            rr = maps[rmap + ar0:rmap + ar1] - rs0
            cc = maps[cmap:cmap + cells[b, 2]]
            assert np.all((rr >= 0) & (rr < rs1 - rs0)) and np.all((cc >= 0) & (cc < cells[c, 3]))
            if kind == 0:
                U = np.where(rr[:, None] >= cc[None, :], U, 0.0)
            np.subtract.at(X, (rr[:, None], cc[None, :]), U)
        if kind == 0:
            S = np.tril(X)
            X = np.linalg.cholesky(S + np.tril(S, -1).T)
        else:
            Ljj = view(d)
            X = np.linalg.solve(np.tril(Ljj), X.T).T
        view(c)[rs0:rs1] = X
    return arena[P.export("sn_csc_map")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_supernodal_device_form_reproduces_oracle(case):
    name, Ap, Ai, Ax, kw = case
    n, P = _plan(case)
    got = _execute_device_form(n, P, Ax)
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lx, info = F.factor(Ax)
    assert info == 0
    assert np.max(np.abs(got - Lx)) <= 1e-12 * np.max(np.abs(Lx)), name
    # off-diagonal slices hold at most 64 rows, every cell fits 128 x 128
    cells = P.export("sn_dev_cells")
    tasks = P.export("sn_dev_tasks")
    off = tasks[:, 0] == 1
    assert np.all(tasks[off, 6] - tasks[off, 5] <= 64)
    assert np.all(cells[:, 2] <= 128) and np.all(cells[:, 3] <= 128)
    # one task per diagonal cell and per slice of each off-diagonal cell
    assert len(tasks) == cells[:, 6].sum()


def _arena_factor(n, P, values):
    """The supernodal factor in its arena (the device form run in numpy)."""
    cells = P.export("sn_dev_cells")
    tasks = P.export("sn_dev_tasks")
    upds = P.export("sn_dev_upds")
    maps = P.export("sn_dev_maps")
    nodes = P.export("sn_nodes")
    arena = np.zeros(int(nodes[-1, 3] + nodes[-1, 1] * nodes[-1, 2]) + 4)
    arena[P.export("sn_value_map")] = values

    def view(c):
        off, ld, h, w = cells[c, :4]
        return np.lib.stride_tricks.as_strided(arena[off:], shape=(h, w), strides=(8, 8 * ld))

    for kind, c, d, ub, ue, rs0, rs1, _ in tasks:
        X = view(c)[rs0:rs1].copy()
        for a, b, ar0, ar1, rmap, cmap, klen in upds[ub:ue]:
            U = view(a)[ar0:ar1] @ view(b).T
            rr = maps[rmap + ar0:rmap + ar1] - rs0
            cc = maps[cmap:cmap + cells[b, 2]]
            if kind == 0:
                U = np.where(rr[:, None] >= cc[None, :], U, 0.0)
            np.subtract.at(X, (rr[:, None], cc[None, :]), U)
        if kind == 0:
            S = np.tril(X)
            X = np.linalg.cholesky(S + np.tril(S, -1).T)
        else:
            X = np.linalg.solve(np.tril(view(d)), X.T).T
        view(c)[rs0:rs1] = X
    return arena, view


def _execute_selinv_form(n, P, arena):
    """Run the supernodal selected-inverse task list (STC_EXPORT_SN_SEL_*) with numpy, as
    the device kernel does: gather the Sigma blocks of each contribution by mode, locate
    rows by searching the source cell's row list, multiply by L's cell, solve with L_JJ,
    and the element recurrence in each diagonal block from the lower part of Z."""
    cells = P.export("sn_dev_cells")
    nodes = P.export("sn_nodes")
    rows = P.export("sn_rows")
    rowoff = P.export("sn_cell_rowoff")
    stasks = P.export("sn_sel_tasks")
    scons = P.export("sn_sel_cons")
    sig = np.zeros_like(arena)

    def view(A, c):
        off, ld, h, w = cells[c, :4]
        return np.lib.stride_tricks.as_strided(A[off:], shape=(h, w), strides=(8, 8 * ld))

    def crow(c):
        return rows[rowoff[c]:rowoff[c] + cells[c, 2]]

    for kind, T, d, cb, ce, rs0, rs1 in stasks:
        J = cells[T, 4]
        w = cells[d, 3]
        Ljj = np.tril(view(arena, d))
        if kind == 0:
            K = cells[T, 5]
            rt = crow(T)[rs0:rs1]
            C = np.zeros((rs1 - rs0, w))
            for lc, sc, mode in scons[cb:ce]:
                Kp = cells[lc, 5]
                rp = crow(lc)
                Sv = view(sig, sc)
                if mode == 0:
                    a = rt - nodes[K, 0]
                    b = rp - nodes[K, 0]
                    G = Sv[np.maximum.outer(a, b), np.minimum.outer(a, b)]
                elif mode == 1:
                    pos = np.searchsorted(crow(sc), rt)
                    assert np.array_equal(crow(sc)[pos], rt)
                    G = Sv[pos[:, None], (rp - nodes[Kp, 0])[None, :]]
                else:
                    pos = np.searchsorted(crow(sc), rp)
                    assert np.array_equal(crow(sc)[pos], rp)
                    G = Sv[pos[None, :], (rt - nodes[K, 0])[:, None]]
                C -= G @ view(arena, lc)
            view(sig, T)[rs0:rs1] = np.linalg.solve(Ljj.T, C.T).T
        else:
            Z = np.zeros((w, w))
            for lc, sc, mode in scons[cb:ce]:
                assert mode == 3 and lc == sc
                Z += view(sig, sc).T @ view(arena, lc)
            Sg = np.zeros((w, w))
            for c in range(w - 1, -1, -1):
                for r in range(w - 1, c, -1):
                    acc = -Z[r, c]
                    for i in range(c + 1, w):
                        acc -= Ljj[i, c] * (Sg[max(r, i), min(r, i)])
                    Sg[r, c] = acc / Ljj[c, c]
                acc = -Z[c, c]
                for i in range(c + 1, w):
                    acc -= Ljj[i, c] * Sg[i, c]
                Sg[c, c] = 1.0 / Ljj[c, c] ** 2 + acc / Ljj[c, c]
            view(sig, d)[:] = np.tril(Sg)
    return sig[P.export("sn_csc_map")]


@pytest.mark.parametrize("case", [c for c in CASES if c[0] != "dense_300"], ids=lambda c: c[0])
def test_supernodal_selinv_form_reproduces_oracle(case):
    # every structural entry of Sigma = A_p^{-1} from the supernodal selected-inverse task
    # list, against the oracle's Takahashi recurrence; a dropped contribution or a wrong
    # mode (transposed source) fails it
    name, Ap, Ai, Ax, kw = case
    n, P = _plan(case)
    arena, _ = _arena_factor(n, P, Ax)
    got = _execute_selinv_form(n, P, arena)
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lx, info = F.factor(Ax)
    So = F.selinv(Lx)
    assert np.max(np.abs(got - So)) <= 1e-11 * np.max(np.abs(So)), name
    modes = P.export("sn_sel_cons")[:, 2]
    if name in ("stcov_nd", "fem3d_nd", "laplace_bordered_nd"):
        assert set(modes.tolist()) >= {0, 1, 2, 3}
