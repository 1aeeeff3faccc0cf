"""GPU parity of the adjoint path: selected inverse, logdet / quadratic-form / solve
gradients, through the C ABI, against the oracle, dense inverses, closed forms and
central finite differences.

Tolerances: Sigma and d logdet / d a on structural entries <= 1e-11 relative to
max |Sigma| (exact recurrences, different summation order); theta-gradients vs the dense
inverse <= 1e-9 relative; vs central differences (h = 1e-6) <= 1e-5 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import api
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def full_sym(n, Ap, Ai, Ax):
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    return (A + sp.tril(A, -1).T).tocsc()


def _selinv_case(P, Ap, Ai, vals):
    fac = P.factorize(dev(vals))
    assert fac.status() == L.STC_OK
    sig = fac.selinv()
    S = sig.to_csc().cpu().numpy()
    g = fac.logdet_backward().cpu().numpy()
    F = O.OracleFactor(P.n, Ap, Ai, P.export("perm"))
    for b in range(vals.shape[0]):
        Lo, _ = F.factor(vals[b])
        So = F.selinv(Lo)
        scale = np.max(np.abs(So))
        assert np.max(np.abs(S[b] - So)) <= 1e-11 * scale, "item %d selinv" % b
        go = F.grad_logdet(So)
        assert np.max(np.abs(g[b] - go)) <= 1e-11 * np.max(np.abs(go)), "item %d grad" % b


@pytest.mark.parametrize("route", ["semisparse", "dense"])
def test_selinv_config1(route):
    vals = []
    for s in range(2):
        Ap, Ai, Ax, coords = I.laplace2d_bordered(seed=s)
        vals.append(Ax)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route=route)
    _selinv_case(P, Ap, Ai, np.stack(vals))


@pytest.mark.parametrize("nb", [8, 16, 32])
def test_selinv_indexed_active_columns(nb):
    n = 301
    Ap, Ai, Ax = I.random_spd(n, 0.01, 4)
    P = Plan(n, Ap, Ai, nb=nb, ordering="rcm", route="semisparse")
    T = P.export("tiles")
    assert np.any((T[:, 0] != T[:, 1]) & (T[:, 4] == 0))
    _selinv_case(P, Ap, Ai, Ax[None])


def test_selinv_band_and_stcov():
    n, bw = 3000, 150
    Ap, Ai = I.band_pattern(n, bw)
    vals = np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(2)])
    P = Plan(n, Ap, Ai, nb=128, ordering="natural", route="semisparse")
    _selinv_case(P, Ap, Ai, vals)
    Ap, Ai, coords = I.stcov_pattern(10, 9, 6, 4)
    th = I.stcov_thetas(2, 7)
    vals = np.stack([I.stcov_values(t, 10, 9, 6, 4) for t in th])
    P = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=32, route="semisparse")
    _selinv_case(P, Ap, Ai, vals)


def test_ar1_selected_inverse_closed_form():
    # Sigma of the unit-innovation AR1 precision is rho^|i-j| / (1 - rho^2)
    nt, rho = 300, 0.8
    Ap, Ai, Ax = I.lower_csc(I.ar1_precision(nt, rho))
    P = Plan(nt, Ap, Ai, nb=16, ordering="natural", route="semisparse")
    S = P.factorize(dev(Ax[None])).selinv().to_csc().cpu().numpy()[0]
    Lp, Li = P.export("Lp"), P.export("Li")
    col = np.repeat(np.arange(nt), np.diff(Lp))
    ref = rho ** np.abs(Li - col) / (1 - rho * rho)
    assert np.max(np.abs(S - ref)) <= 1e-11 * np.max(ref)


def _theta_objective_grad(P, Ap, Ai, thetas, x, dims):
    """d/dtheta [logdet Q(theta) - x^T Q(theta) x] through the GPU adjoint."""
    nx, ny, nt, nbd = dims
    vals = np.stack([I.stcov_values(t, nx, ny, nt, nbd) for t in thetas])
    fac = P.factorize(dev(vals))
    gl = fac.logdet_backward()
    gq = torch.empty_like(gl)
    xs = dev(x)
    assert L.stc_sym_outer_backward(P.h, len(thetas), xs, xs, None, gq, 0) == L.STC_OK
    g = (gl - gq).cpu().numpy()
    ld = fac.logdet().cpu().numpy()
    q = torch.empty(len(thetas), dtype=torch.float64, device="cuda")
    assert L.stc_quad_form(P.h, len(thetas), dev(vals), xs, q) == L.STC_OK
    f = ld - q.cpu().numpy()
    dth = np.stack([I.stcov_dtheta(t, nx, ny, nt, nbd) @ g[b] for b, t in enumerate(thetas)])
    return f, dth, vals


def test_theta_gradient_downsized_config5():
    # 20x20x10 field + 20 border rows (n = 4,020), 3 theta draws, fixed x ~ N(0, I)
    dims = (20, 20, 10, 20)
    Ap, Ai, coords = I.stcov_pattern(*dims)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
    thetas = I.stcov_thetas(3, 11)
    x = np.stack([I.rhs(n, 100 + b)[0] for b in range(3)])
    f, dth, vals = _theta_objective_grad(P, Ap, Ai, thetas, x, dims)
    for b, t in enumerate(thetas):
        Q = full_sym(n, Ap, Ai, vals[b]).toarray()
        Qi = np.linalg.inv(Q)
        dQ = I.stcov_dtheta(t, *dims)
        ref = np.empty(3)
        for k in range(3):
            M = full_sym(n, Ap, Ai, dQ[k]).toarray()
            ref[k] = np.sum(Qi * M) - x[b] @ M @ x[b]
        assert np.max(np.abs(dth[b] - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-9, (dth[b], ref)
        s, ldref = np.linalg.slogdet(Q)
        assert abs(f[b] - (ldref - x[b] @ Q @ x[b])) <= 1e-10 * abs(ldref)
    # central finite differences on theta through the GPU forward (h = 1e-6)
    h = 1e-6
    b = 1
    for k in range(3):
        tp, tm = thetas[b].copy(), thetas[b].copy()
        tp[k] += h
        tm[k] -= h
        fp, _, _ = _theta_objective_grad(P, Ap, Ai, tp[None], x[b:b + 1], dims)
        fm, _, _ = _theta_objective_grad(P, Ap, Ai, tm[None], x[b:b + 1], dims)
        fd = (fp[0] - fm[0]) / (2 * h)
        assert abs(fd - dth[b, k]) <= 1e-5 * max(1.0, abs(dth[b, k])), (k, fd, dth[b, k])


def test_theta_gradient_closed_form_without_border():
    # border-free: d/dtau = n/tau, d/drho = -nx ny 2 rho/(1-rho^2),
    # d/dkappa = nt [ny sum_a 2k/(k2+mu_a) + nx sum_b 2k/(k2+mu_b)]
    dims = (14, 12, 8, 0)
    nx, ny, nt, _ = dims
    Ap, Ai, coords = I.stcov_pattern(*dims)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=32, route="semisparse")
    thetas = np.array([[2.0, 0.6, 0.7], [0.3, 0.9, 1.5]])
    x = np.zeros((2, n))
    _, dth, _ = _theta_objective_grad(P, Ap, Ai, thetas, x, dims)
    for b, (tau, rho, kap) in enumerate(thetas):
        mux = 2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
        muy = 2 - 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
        k2 = kap * kap
        ref = [n / tau, -nx * ny * 2 * rho / (1 - rho * rho),
               nt * (ny * np.sum(2 * kap / (k2 + mux)) + nx * np.sum(2 * kap / (k2 + muy)))]
        assert np.allclose(dth[b], ref, rtol=1e-10, atol=1e-9), (dth[b], ref)


def test_autograd_logdet_quad_solve():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(12, 12, 2)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=32)
    v0 = dev(np.stack([Ax, Ax * 1.1]))
    dv = dev(np.stack([np.abs(Ax) * 0.01, np.abs(Ax) * 0.02]))
    x = dev(np.stack([I.rhs(n, 1)[0], I.rhs(n, 2)[0]]))
    b = dev(np.stack([I.rhs(n, 3)[0], I.rhs(n, 4)[0]]))
    t = torch.zeros(1, dtype=torch.float64, device="cuda", requires_grad=True)

    def obj(tt):
        v = v0 + tt * dv
        return (api.logdet(v, P) - api.quad_form(v, x, P) + (api.solve(v, b, P) * b).sum(dim=1)).sum()

    f = obj(t)
    f.backward()
    h = 1e-6
    with torch.no_grad():
        fd = (obj(torch.full_like(t, h)) - obj(torch.full_like(t, -h))) / (2 * h)
    assert abs(t.grad.item() - fd.item()) <= 1e-5 * max(1.0, abs(fd.item()))


def test_quad_form_and_outer_backward_vs_numpy():
    Ap, Ai, Ax = I.random_spd(200, 0.03, 9)
    n = 200
    P = Plan(n, Ap, Ai, nb=16)
    x = np.stack([I.rhs(n, 5)[0], I.rhs(n, 6)[0]])
    vals = np.stack([Ax, 2 * Ax])
    q = torch.empty(2, dtype=torch.float64, device="cuda")
    assert L.stc_quad_form(P.h, 2, dev(vals), dev(x), q) == L.STC_OK
    g = torch.empty(2, len(Ai), dtype=torch.float64, device="cuda")
    sc = dev(np.array([1.0, -0.5]))
    assert L.stc_sym_outer_backward(P.h, 2, dev(x), dev(x), sc, g, 0) == L.STC_OK
    gq = torch.empty_like(g)
    assert L.stc_quad_backward(P.h, 2, dev(x), sc, gq, 0) == L.STC_OK    # u = v = x form
    assert torch.equal(gq, g)
    col = np.repeat(np.arange(n), np.diff(Ap))
    for bb in range(2):
        A = full_sym(n, Ap, Ai, vals[bb])
        assert abs(q[bb].item() - x[bb] @ (A @ x[bb])) <= 1e-12 * abs(x[bb] @ (A @ x[bb]))
        ref = sc[bb].item() * np.where(Ai == col, 1.0, 2.0) * x[bb][Ai] * x[bb][col]
        assert np.allclose(g[bb].cpu().numpy(), ref, rtol=1e-14, atol=1e-14)
