"""GPU parity of the supernodal route (Sec. 5.4) through the C ABI against the oracle.

Plans analysed with route="supernodal" store L in the non-uniform supernodal panels
and factorize with the supernodal device kernels (scattered updates through
sorted-subset row and column maps, POTRF and panel TRSM per cell); logdet, solve and the
CSC export read that layout.  Tolerances are those of test_gpu_factor.py.  The
persistent kernels walk a topological queue, so the serial replay (one CTA) is the
reference schedule: parallel grids must reproduce it bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan
from test_gpu_factor import check_against_oracle, dev
from test_supernodal import CASES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(Ap, Ai, Ax, count, seed):
    """Item 0 is Ax; item b scales every off-diagonal entry by one factor s_b in [0.3, 1],
    i.e. (1 - s_b) D + s_b A, a convex combination of SPD matrices, so it stays SPD."""
    n = len(Ap) - 1
    col = np.repeat(np.arange(n), np.diff(Ap))
    off = Ai != col
    rng = np.random.default_rng(seed)
    return np.stack([Ax] + [np.where(off, Ax * rng.uniform(0.3, 1.0), Ax) for _ in range(count - 1)])


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_supernodal_route_parity(case):
    name, Ap, Ai, Ax, kw = case
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, route="supernodal", **kw)
    assert P.route == "supernodal"
    vals = _batch(Ap, Ai, Ax, 3, 1)
    rhs = np.random.default_rng(2).standard_normal((3, 2, n))
    check_against_oracle(P, Ap, Ai, vals, rhs)


@pytest.mark.parametrize("seed", range(6))
def test_supernodal_random_patterns(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(20, 600))
    Ap, Ai, Ax = I.random_spd(n, float(rng.uniform(0.003, 0.05)), 40 + seed)
    ordering = ["rcm", "natural", "given"][seed % 3]
    perm = rng.permutation(n) if ordering == "given" else None
    P = Plan(n, Ap, Ai, route="supernodal", ordering=ordering if perm is None else "auto", perm=perm)
    batch = int(rng.integers(1, 4))
    check_against_oracle(P, Ap, Ai, _batch(Ap, Ai, Ax, batch, seed), rng.standard_normal((batch, 1, n)))


def test_supernodal_spatio_temporal_with_border():
    Ap, Ai, coords = I.stcov_pattern(14, 12, 8, 6)
    th = I.stcov_thetas(3, 100)
    vals = np.stack([I.stcov_values(t, 14, 12, 8, 6) for t in th])
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, route="supernodal")
    check_against_oracle(P, Ap, Ai, vals, np.stack([I.rhs(n, s, 1) for s in range(3)]))


def test_supernodal_matches_tile_route_logdet_and_storage():
    # same ordering, same symbolic factor: the supernodal and the tile routes give the
    # same factor up to summation order, and the supernodal panels store fewer entries
    Ap, Ai, Ax, coords = I.fem3d(12, 11, 10)
    n = len(Ap) - 1
    Ps = Plan(n, Ap, Ai, coords=coords, nb=32, route="supernodal", nd_leaf=32)
    Pt = Plan(n, Ap, Ai, coords=coords, nb=32, route="semisparse", nd_leaf=32)
    assert np.array_equal(Ps.export("perm"), Pt.export("perm"))
    assert Ps.info["stored_entries"] < Pt.info["stored_entries"]
    v = dev(Ax[None])
    Ls = Ps.factorize(v).to_csc().cpu().numpy()
    Lt = Pt.factorize(v).to_csc().cpu().numpy()
    assert np.max(np.abs(Ls - Lt)) <= 1e-13 * np.max(np.abs(Lt))


def test_supernodal_not_spd_item_reports_info():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(seed=0)
    n = len(Ap) - 1
    vals = np.stack([I.laplace2d_bordered(seed=s)[2] for s in range(3)])
    col = np.repeat(np.arange(n), np.diff(Ap))
    diag = np.nonzero(Ai == col)[0]
    vals[1, diag[300]] = -5.0
    P = Plan(n, Ap, Ai, coords=coords, route="supernodal")
    fac = P.factorize(dev(vals))
    assert fac.status() == L.STC_OK
    info = fac.info.cpu().numpy()
    ld = fac.logdet().cpu().numpy()
    _, oinfo = O.OracleFactor(n, Ap, Ai, P.export("perm")).factor(vals[1])
    assert oinfo > 0 and info[1] == oinfo and info[0] == 0 and info[2] == 0
    assert np.isnan(ld[1]) and np.isfinite(ld[0]) and np.isfinite(ld[2])


def test_supernodal_serial_and_parallel_replay_bit_identical():
    Ap, Ai, coords = I.stcov_pattern(14, 12, 8, 6)
    vals = np.stack([I.stcov_values(t, 14, 12, 8, 6) for t in I.stcov_thetas(4, 7)])
    n = len(Ap) - 1
    v = dev(vals)
    b = dev(np.random.default_rng(3).standard_normal((4, 2, n)))
    out = {}
    for ctas in (1, 0, 3 * 152):
        P = Plan(n, Ap, Ai, coords=coords, route="supernodal", replay_ctas=ctas)
        fac = P.factorize(v)
        assert fac.status() == L.STC_OK
        out[ctas] = (fac.data.clone(), fac.logdet(), fac.solve(b))
    for ctas in (0, 3 * 152):
        for a, r in zip(out[ctas], out[1]):
            assert torch.equal(a, r)


def test_supernodal_refuses_the_allocation_free_entry():
    Ap, Ai, _ = I.tridiag(200, 0)
    P = Plan(200, Ap, Ai, route="supernodal", ordering="natural")
    P.upload()
    fac = torch.zeros(P.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
    v = torch.zeros(1, P.nnzA, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.stc_factorize_noalloc(P.h, v, 1, fac, info) == L.STC_ERR_UNSUPPORTED


@pytest.mark.parametrize("case", [c for c in CASES if c[0] != "dense_300"], ids=lambda c: c[0])
def test_supernodal_selinv_and_logdet_gradient(case):
    # Sigma on every structural entry and d logdet / d a against the oracle (Takahashi),
    # with the tolerances of test_gpu_adjoint.py
    from test_gpu_adjoint import _selinv_case
    name, Ap, Ai, Ax, kw = case
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, route="supernodal", **kw)
    _selinv_case(P, Ap, Ai, _batch(Ap, Ai, Ax, 2, 5))


def test_supernodal_selinv_spatio_temporal_and_serial_replay():
    from test_gpu_adjoint import _selinv_case
    Ap, Ai, coords = I.stcov_pattern(14, 12, 8, 6)
    vals = np.stack([I.stcov_values(t, 14, 12, 8, 6) for t in I.stcov_thetas(3, 9)])
    n = len(Ap) - 1
    _selinv_case(Plan(n, Ap, Ai, coords=coords, route="supernodal"), Ap, Ai, vals)
    out = []
    for ctas in (1, 0):
        P = Plan(n, Ap, Ai, coords=coords, route="supernodal", replay_ctas=ctas)
        fac = P.factorize(dev(vals))
        out.append((fac.selinv().data.clone(), fac.logdet_backward().clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
