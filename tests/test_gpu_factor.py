"""GPU parity: factorize / logdet / solve through the C ABI against the CPU oracle.

Tolerances (FP64 throughout; the factor bound is the forward error of two exact
Cholesky factorizations that differ only in summation order, ~kappa * c * u * |L|):
  * factor entries: |L_gpu - L_oracle| <= 1e-11 * max |L_:j| per column (two exact
    factorizations differing only in summation order);
  * residual ||L L^T - A_p||_F / ||A_p||_F <= 1e-12 (the spec gate);
  * logdet relative error <= 1e-10, solve relative error <= 1e-10;
  * the dense and semisparse routes agree entrywise to <= 1e-13 (relative to max |L|).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_L = 1e-11
TOL_RES = 1e-12
TOL_LD = 1e-10
TOL_X = 1e-10


def full_sym(n, Ap, Ai, Ax):
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    return (A + sp.tril(A, -1).T).tocsc()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def check_against_oracle(P, Ap, Ai, vals, rhs=None):
    """vals [batch, nnzA]; returns the GPU results after asserting parity per item."""
    n = P.n
    fac = P.factorize(dev(vals))
    assert fac.status() == L.STC_OK
    Lx = fac.to_csc().cpu().numpy()
    ld = fac.logdet().cpu().numpy()
    info = fac.info.cpu().numpy()
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    assert np.array_equal(P.export("Lp"), F.Lp) and np.array_equal(P.export("Li"), F.Li)
    x = None
    if rhs is not None:
        x = fac.solve(dev(rhs)).cpu().numpy()
    col = np.repeat(np.arange(n), np.diff(F.Lp))
    for b in range(vals.shape[0]):
        Lo, oinfo = F.factor(vals[b])
        assert info[b] == oinfo == 0
        scale = np.maximum.reduceat(np.abs(Lo), F.Lp[:-1])[col]
        err = np.abs(Lx[b] - Lo) / scale
        assert err.max() <= TOL_L, "item %d: factor entry error %.3e" % (b, err.max())
        Lm = sp.csc_matrix((Lx[b], F.Li, F.Lp), shape=(n, n))
        Apm = full_sym(n, Ap, Ai, vals[b])[F.perm][:, F.perm]
        res = sp.linalg.norm(Lm @ Lm.T - Apm) / sp.linalg.norm(Apm)
        assert res <= TOL_RES, "item %d: residual %.3e" % (b, res)
        ldo = F.logdet(Lo)
        assert abs(ld[b] - ldo) <= TOL_LD * abs(ldo), "item %d: logdet %r vs %r" % (b, ld[b], ldo)
        if rhs is not None:
            for r in range(rhs.shape[1]):
                xo = F.solve(Lo, rhs[b, r])
                e = np.linalg.norm(x[b, r] - xo) / np.linalg.norm(xo)
                assert e <= TOL_X, "item %d rhs %d: solve error %.3e" % (b, r, e)
    return fac, Lx, ld, x


def c1_batch(batch):
    vals = []
    for s in range(batch):
        Ap, Ai, Ax, coords = I.laplace2d_bordered(seed=s)
        vals.append(Ax)
    return Ap, Ai, coords, np.stack(vals)


@pytest.mark.parametrize("route", ["semisparse", "dense"])
@pytest.mark.parametrize("batch", [1, 3])
def test_config1_factor_logdet_solve(route, batch):
    Ap, Ai, coords, vals = c1_batch(batch)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route=route)
    rhs = np.stack([I.rhs(n, 1 + b, 2) for b in range(batch)])
    check_against_oracle(P, Ap, Ai, vals, rhs)


@pytest.mark.parametrize("nb", [8, 16, 32, 64])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_indexed_active_columns(nb, seed):
    n = 517 + 13 * seed   # ragged last tile
    Ap, Ai, Ax = I.random_spd(n, 0.006, seed)
    P = Plan(n, Ap, Ai, nb=nb, ordering="rcm", route="semisparse")
    T = P.export("tiles")
    off = T[:, 0] != T[:, 1]
    assert np.any(T[off, 4] == 0), "want non-contiguous active-column tiles"
    vals = np.stack([Ax, Ax * (1 + 0.01 * np.random.default_rng(9).uniform(size=len(Ax)))])
    rhs = np.stack([I.rhs(n, 7, 1), I.rhs(n, 8, 1)])
    check_against_oracle(P, Ap, Ai, vals, rhs)


@pytest.mark.parametrize("slices", [1, 2, 4, 8])
def test_band_row_slices(slices):
    n, bw = 5000, 200   # 39 full tiles of 128 + a ragged tile of 8 rows
    Ap, Ai = I.band_pattern(n, bw)
    vals = np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(2)])
    P = Plan(n, Ap, Ai, nb=128, ordering="natural", route="semisparse", row_slices=slices)
    check_against_oracle(P, Ap, Ai, vals, np.stack([I.rhs(n, s, 1) for s in range(2)]))


@pytest.mark.parametrize("n,bw,nb,slices", [(3000, 40, 128, 8), (2001, 70, 128, 8), (1500, 14, 64, 8),
                                             (999, 200, 64, 8), (5000, 200, 128, 2)])
def test_row_sliced_diagonal_factorization(n, bw, nb, slices):
    # POTRF(k) partitioned over the row slices of (k,k): each slice solves its rows against
    # the column groups the earlier slices publish, then factors its own block.  Bands
    # narrower than n_b make banded diagonal tiles in which a slice skips the groups lying
    # wholly outside its rows' band; the exported task list shows that this happens.
    Ap, Ai = I.band_pattern(n, bw)
    vals = np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(2)])
    P = Plan(n, Ap, Ai, nb=nb, ordering="natural", route="semisparse", row_slices=slices)
    T = L.stc_plan_export_taskset(P.h, slices, False, L.STC_TASKSET_TASKS).reshape(-1, 13)
    tiles = L.stc_plan_export_taskset(P.h, slices, False, L.STC_TASKSET_TILES).reshape(-1, 13)
    sy = T[T[:, 0] == 2]
    assert len(sy) and (sy[:, 10] > 0).any(), "no diagonal tile factored by several slices"
    if bw + 16 < nb:
        kd = tiles[sy[:, 1], 7]
        assert (sy[:, 5] - kd >= 16).any(), "no slice skips a column group"
    check_against_oracle(P, Ap, Ai, vals, np.stack([I.rhs(n, 20 + s, 1) for s in range(2)]))


def test_stcov_small_with_border():
    Ap, Ai, coords = I.stcov_pattern(14, 12, 8, 6)
    th = I.stcov_thetas(3, 100)
    vals = np.stack([I.stcov_values(t, 14, 12, 8, 6) for t in th])
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=32, route="semisparse")
    check_against_oracle(P, Ap, Ai, vals, np.stack([I.rhs(n, s, 1) for s in range(3)]))


def test_fem3d_small_dense_route():
    Ap, Ai, Ax, coords = I.fem3d(12, 11, 10)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=32, route="dense", nd_leaf=32)
    check_against_oracle(P, Ap, Ai, Ax[None], I.rhs(n, 3, 1)[None])


def test_route_equivalence_dense_vs_semisparse():
    Ap, Ai, coords, vals = c1_batch(2)
    n = len(Ap) - 1
    Pd = Plan(n, Ap, Ai, coords=coords, nb=64, route="dense")
    Ps = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
    assert np.array_equal(Pd.export("perm"), Ps.export("perm"))
    Ld = Pd.factorize(dev(vals)).to_csc().cpu().numpy()
    Ls = Ps.factorize(dev(vals)).to_csc().cpu().numpy()
    assert np.max(np.abs(Ld - Ls)) <= 1e-13 * np.max(np.abs(Ld))


def test_deterministic_repeat():
    n, bw = 3000, 150
    Ap, Ai = I.band_pattern(n, bw)
    v = dev(np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(4)]))
    P = Plan(n, Ap, Ai, nb=64, ordering="natural", route="semisparse")
    a = P.factorize(v).data.clone()
    b = P.factorize(v).data.clone()
    assert torch.equal(a, b)


def test_not_spd_item_reports_info_and_nan_logdet():
    Ap, Ai, coords, vals = c1_batch(3)
    n = len(Ap) - 1
    bad = vals[1].copy()
    col = np.repeat(np.arange(n), np.diff(Ap))
    diag = np.nonzero(Ai == col)[0]
    bad[diag[500]] = -5.0
    vals[1] = bad
    P = Plan(n, Ap, Ai, coords=coords, nb=64)
    fac = P.factorize(dev(vals))
    assert fac.status() == L.STC_OK
    info = fac.info.cpu().numpy()
    ld = fac.logdet().cpu().numpy()
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    _, oinfo = F.factor(bad)
    assert oinfo > 0 and info[1] == oinfo
    assert info[0] == 0 and info[2] == 0
    assert np.isnan(ld[1]) and np.isfinite(ld[0]) and np.isfinite(ld[2])


def test_wait_limit_reports_timeout_and_context_survives():
    n, bw = 20000, 200
    Ap, Ai = I.band_pattern(n, bw)
    v = dev(I.band_values(n, bw, 0, Ap, Ai)[None])
    P = Plan(n, Ap, Ai, nb=128, ordering="natural", spin_limit=1, row_slices=1)
    fac = P.factorize(v)
    assert fac.status() == L.STC_ERR_TIMEOUT
    # the context is still usable: an unlimited plan on the same pattern is exact
    P2 = Plan(n, Ap, Ai, nb=128, ordering="natural")
    fac2 = P2.factorize(v)
    assert fac2.status() == L.STC_OK
    F = O.OracleFactor(n, Ap, Ai)
    Lo, _ = F.factor(v[0].cpu().numpy())
    ld = fac2.logdet().cpu().numpy()[0]
    assert abs(ld - F.logdet(Lo)) <= TOL_LD * abs(F.logdet(Lo))


def test_invalid_device_arguments():
    Ap, Ai, _ = I.tridiag(50, 0)
    P = Plan(50, Ap, Ai, nb=8)
    x = torch.zeros(1, P.nnzA, dtype=torch.float64, device="cuda")
    f = torch.zeros(P.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
    w = torch.zeros(P.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.stc_factorize(P.h, x, 0, f, w, info) == L.STC_ERR_INVALID_ARG
    assert L.lib().stc_factorize(P.h, None, 1, None, None, None, None) == L.STC_ERR_INVALID_ARG
    b = torch.zeros(1, 1, 50, dtype=torch.float64, device="cuda")
    assert L.stc_solve(P.h, f, 1, 1, b, b, w) == L.STC_ERR_INVALID_ARG


def test_loaded_plan_factorizes_identically():
    # a plan saved and loaded again (stc_plan_save / stc_plan_load) holds the same arrays,
    # so its factors are bit-identical to the original plan's
    Ap, Ai, coords, vals = c1_batch(2)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64)
    Q = Plan.load(P.save())
    a = P.factorize(dev(vals))
    b = Q.factorize(dev(vals))
    assert b.status() == L.STC_OK
    assert torch.equal(a.data, b.data)
    assert torch.equal(a.logdet(), b.logdet())


def test_null_workspace_uses_the_plans_own():
    # d_work == NULL (and d_sigma == NULL in logdet_backward) runs on buffers owned by the
    # plan; results are bit-identical to the caller-owned ones
    Ap, Ai, coords, vals = c1_batch(3)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64)
    assert L.stc_plan_sync_status(P.h) == L.STC_ERR_INVALID_ARG   # not used yet
    v = dev(vals)
    ref = P.factorize(v)
    fac = torch.empty_like(ref.data)
    info = torch.empty(3, dtype=torch.int32, device="cuda")
    assert L.stc_factorize(P.h, v, 3, fac, None, info) == L.STC_OK
    assert L.stc_plan_sync_status(P.h) == L.STC_OK
    assert torch.equal(fac, ref.data) and torch.equal(info, ref.info)
    b = dev(np.random.default_rng(4).standard_normal((3, 2, n)))
    x = torch.empty_like(b)
    assert L.stc_solve(P.h, fac, 3, 2, b, x, None) == L.STC_OK
    assert torch.equal(x, ref.solve(b))
    g = torch.empty(3, P.nnzA, dtype=torch.float64, device="cuda")
    assert L.stc_logdet_backward(P.h, fac, 3, None, g, 0, None, None) == L.STC_OK
    assert L.stc_plan_sync_status(P.h) == L.STC_OK
    assert torch.equal(g, ref.logdet_backward())


def _fused_cases():
    n, bw = 5000, 200
    Ap, Ai = I.band_pattern(n, bw)
    vals = np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(3)])
    yield "band n=5000 bw 200", (n, Ap, Ai), dict(nb=128, ordering="natural", route="semisparse"), vals
    n2, bw2 = 3000, 40
    Ap2, Ai2 = I.band_pattern(n2, bw2)
    vals2 = np.stack([I.band_values(n2, bw2, s, Ap2, Ai2) for s in range(20)])
    yield "band n=3000 bw 40, 20 value sets", (n2, Ap2, Ai2), dict(nb=128, ordering="natural", route="semisparse"), vals2
    Ap3, Ai3, coords, vals3 = c1_batch(2)
    yield "config 1, dense route", (len(Ap3) - 1, Ap3, Ai3), dict(coords=coords, nb=64, route="dense"), vals3
    n4 = 517
    Ap4, Ai4, Ax4 = I.random_spd(n4, 0.006, 1)
    yield "random indexed, n_b 16", (n4, Ap4, Ai4), dict(nb=16, ordering="rcm", route="semisparse"), Ax4[None]
    yield "config 1, supernodal route", (len(Ap3) - 1, Ap3, Ai3), dict(coords=coords, nb=64, route="supernodal"), vals3


@pytest.mark.parametrize("case", list(_fused_cases()), ids=lambda c: c[0])
def test_factorize_solve_fused(case):
    # factorization + solve in one call (the forward substitution inside the factorization
    # launch): the factor equals stc_factorize's to the bit, x matches the oracle's solve
    name, (n, Ap, Ai), kw, vals = case
    batch = vals.shape[0]
    P = Plan(n, Ap, Ai, **kw)
    rhs = np.stack([I.rhs(n, 30 + b, 2) for b in range(batch)])
    fac1 = P.factorize(dev(vals))
    fac2, x = P.factorize_solve(dev(vals), dev(rhs), check_status=True)
    assert int(fac2.info.abs().sum()) == 0
    assert torch.equal(fac1.data, fac2.data), name
    x = x.cpu().numpy()
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    for b in sorted({0, batch - 1}):
        Lo, _ = F.factor(vals[b])
        for r in range(2):
            xo = F.solve(Lo, rhs[b, r])
            assert np.linalg.norm(x[b, r] - xo) <= TOL_X * np.linalg.norm(xo), (name, b, r)
    # a second call on the same workspace gives the same x
    _, x2 = P.factorize_solve(dev(vals), dev(rhs))
    assert np.array_equal(x2.cpu().numpy(), x)


@pytest.mark.parametrize("case", [c for c in _fused_cases() if c[0] in (
    "band n=5000 bw 200", "random indexed, n_b 16", "config 1, supernodal route")], ids=lambda c: c[0])
def test_factorize_solve_pinned_host_inputs(case):
    # values and right-hand sides left in pinned host memory and read in place by the
    # kernels (value upload inside the launch, the scatter kernel, or the supernodal
    # route's separate calls): the same factor and solution, to the bit, as from HBM
    name, (n, Ap, Ai), kw, vals = case
    P = Plan(n, Ap, Ai, **kw)
    rhs = np.stack([I.rhs(n, 60 + b, 2) for b in range(vals.shape[0])])
    fac1, x1 = P.factorize_solve(dev(vals), dev(rhs))
    hv = torch.from_numpy(np.ascontiguousarray(vals)).pin_memory()
    hb = torch.from_numpy(np.ascontiguousarray(rhs)).pin_memory()
    fac2, x2 = P.factorize_solve(hv, hb, check_status=True)
    assert int(fac2.info.abs().sum()) == 0
    assert torch.equal(fac1.data, fac2.data), name
    assert torch.equal(x1, x2), name
