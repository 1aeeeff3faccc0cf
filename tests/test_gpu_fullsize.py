"""Full-size parity on the benchmark workloads, in the launch configuration bench.py times.

At these sizes the oracle is too slow for every output, so the checks are
  * config 2 (n = 200,000 band, batch 64): two sampled items element by element against
    the oracle; every item's solve residual and info;
  * config 3 (60x60x50 spatio-temporal, n = 180,000 field): the closed-form logdet and
    theta-gradient of the border-free precision; with the 20 border rows, solve
    residuals;
  * config 4 (64^3 FEM, dense route): the closed-form logdet of the unit-conductance
    Neumann Laplacian; lognormal conductances: solve residual; the mixed batch
    32^3 / 48^3 / 64^3 x 8 in one launch: residuals and a sampled oracle logdet.
Tolerances as in test_gpu_factor.py (logdet 1e-10, solve 1e-10, factor entries 1e-11).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Factor, Group, Plan

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def full_sym(n, Ap, Ai, Ax):
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    return (A + sp.tril(A, -1).T).tocsr()


def item(fac, b):
    fd = fac.plan.info["factor_doubles"]
    return Factor(fac.plan, fac.data[b * fd:(b + 1) * fd], fac.info[b:b + 1], 1)


def residual(n, Ap, Ai, Ax, x, b):
    A = full_sym(n, Ap, Ai, Ax)
    return np.linalg.norm(A @ x - b) / np.linalg.norm(b)


def test_config2_band_batch64():
    n, bw, batch = 200_000, 200, 64
    Ap, Ai = I.band_pattern(n, bw)
    P = Plan(n, Ap, Ai, nb=128, ordering="natural", route="semisparse")
    vals = torch.empty(batch, P.nnzA, dtype=torch.float64, device="cuda")
    host = {}
    for s in range(batch):
        v = I.band_values(n, bw, s, Ap, Ai)
        vals[s].copy_(torch.from_numpy(v))
        if s in (0, 37, batch - 1):
            host[s] = v
    rhs = np.stack([I.rhs(n, 1000 + s)[0] for s in range(batch)])
    fac = P.factorize(vals)
    x = fac.solve(dev(rhs)[:, None, :]).cpu().numpy()[:, 0]
    ld = fac.logdet().cpu().numpy()
    assert fac.status() == L.STC_OK and int(fac.info.abs().sum()) == 0
    assert np.all(np.isfinite(ld))
    F = O.OracleFactor(n, Ap, Ai)
    col = np.repeat(np.arange(n), np.diff(F.Lp))
    for s, v in host.items():
        assert residual(n, Ap, Ai, v, x[s], rhs[s]) <= 1e-10
        if s == 37:
            continue
        Lo, info = F.factor(v)
        assert info == 0
        Lg = item(fac, s).to_csc().cpu().numpy()[0]
        scale = np.maximum.reduceat(np.abs(Lo), F.Lp[:-1])[col]
        assert np.max(np.abs(Lg - Lo) / scale) <= 1e-11
        assert abs(ld[s] - F.logdet(Lo)) <= 1e-10 * abs(F.logdet(Lo))
        xo = F.solve(Lo, rhs[s])
        assert np.linalg.norm(x[s] - xo) <= 1e-10 * np.linalg.norm(xo)


def test_config3_closed_form_logdet_and_theta_gradient():
    nx, ny, nt = 60, 60, 50
    Ap, Ai, coords = I.stcov_pattern(nx, ny, nt, 0)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
    thetas = np.array([[3.0, 0.8, 0.3], [0.2, 0.1, 1.7]])
    vals = np.stack([I.stcov_values(t, nx, ny, nt, 0) for t in thetas])
    fac = P.factorize(dev(vals))
    ld = fac.logdet().cpu().numpy()
    g = fac.logdet_backward().cpu().numpy()
    assert fac.status() == L.STC_OK
    mux = 2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
    muy = 2 - 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
    for b, (tau, rho, kap) in enumerate(thetas):
        k2 = kap * kap
        ref = n * np.log(tau) + nx * ny * np.log(1 - rho * rho) + nt * (
            ny * np.sum(np.log(k2 + mux)) + nx * np.sum(np.log(k2 + muy)))
        assert abs(ld[b] - ref) <= 1e-10 * abs(ref)
        dth = I.stcov_dtheta(thetas[b], nx, ny, nt, 0) @ g[b]
        gref = [n / tau, -nx * ny * 2 * rho / (1 - rho * rho),
                nt * (ny * np.sum(2 * kap / (k2 + mux)) + nx * np.sum(2 * kap / (k2 + muy)))]
        assert np.allclose(dth, gref, rtol=1e-9, atol=1e-7), (dth, gref)


def test_config3_with_border_solve_residual():
    Ap, Ai, coords = I.stcov_pattern()
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
    thetas = I.stcov_thetas(2, 0)
    vals = np.stack([I.stcov_values(t) for t in thetas])
    rhs = np.stack([I.rhs(n, 50 + b)[0] for b in range(2)])
    fac = P.factorize(dev(vals))
    x = fac.solve(dev(rhs)).cpu().numpy()
    assert fac.status() == L.STC_OK and int(fac.info.abs().sum()) == 0
    for b in range(2):
        assert residual(n, Ap, Ai, vals[b], x[b], rhs[b]) <= 1e-10


def test_config4_fem64_dense_route():
    m = 64
    Ap, Ai, Ax1, coords = I.fem3d(m, m, m, unit_conductance=True)
    _, _, Ax, _ = I.fem3d(m, m, m, seed=0)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route="dense")
    assert P.route == "dense"
    fac = P.factorize(dev(np.stack([Ax1, Ax])))
    ld = fac.logdet().cpu().numpy()
    b = I.rhs(n, 9, 2)
    x = fac.solve(dev(b)).cpu().numpy()
    e = 2 - 2 * np.cos(np.pi * np.arange(m) / m)
    lam = e[:, None, None] + e[None, :, None] + e[None, None, :] + 1e-3
    ref = np.sum(np.log(lam))
    assert abs(ld[0] - ref) <= 1e-10 * abs(ref)
    assert residual(n, Ap, Ai, Ax1, x[0], b[0]) <= 1e-10
    assert residual(n, Ap, Ai, Ax, x[1], b[1]) <= 1e-10


def test_config4_mixed_batch_one_launch():
    plans, vals, pats = [], [], []
    for m in (32, 48, 64):
        vs = []
        for s in range(8):
            Ap, Ai, Ax, coords = I.fem3d(m, m, m, seed=s)
            vs.append(Ax)
        n = len(Ap) - 1
        pats.append((n, Ap, Ai, vs))
        plans.append(Plan(n, Ap, Ai, coords=coords, nb=64, route="dense"))
        vals.append(dev(np.stack(vs)))
    G = Group(plans, [8, 8, 8])
    facs = G.factorize(vals)
    assert G.status() == L.STC_OK
    for (n, Ap, Ai, vs), f in zip(pats, facs):
        assert int(f.info.abs().sum()) == 0
        b = I.rhs(n, 3, 8)
        x = f.solve(dev(b)).cpu().numpy()
        for s in (0, 7):
            assert residual(n, Ap, Ai, vs[s], x[s], b[s]) <= 1e-10
    n, Ap, Ai, vs = pats[0]
    F = O.OracleFactor(n, Ap, Ai, plans[0].export("perm"))
    Lo, _ = F.factor(vs[5])
    ld = facs[0].logdet().cpu().numpy()[5]
    assert abs(ld - F.logdet(Lo)) <= 1e-10 * abs(F.logdet(Lo))
