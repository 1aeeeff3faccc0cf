"""GPU edge cases and the race check, through the C ABI against the CPU oracle.

Degenerate sizes and structures (n = 1, n < n_b: a single ragged tile, n a multiple of
n_b, a diagonal matrix, a dense matrix, an arrowhead with its dense rows last,
disconnected blocks) on the three routes, with the tolerances of test_gpu_factor.py.

Race check: the persistent kernels walk a topological task queue, so one CTA executing
it in queue order (replay_ctas = 1) is a schedule with no concurrency at all.  Every
update into a tile runs in a fixed order whatever the schedule, so a parallel run (the
default grid, and a grid larger than the GPU holds at once) must reproduce the serial
run bit for bit: factor storage, log-determinants, solves and the selected inverse.  A
missing dependency wait or a missing fence would let a parallel run read stale data and
break the equality.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan
from test_gpu_factor import check_against_oracle, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _spd_from_pattern(n, rows, cols, seed):
    rng = np.random.default_rng(seed)
    M = sp.coo_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, n)).tocsc()
    M = M + M.T
    M = M + sp.diags(np.asarray(abs(M).sum(axis=1)).ravel() + 1.0)
    return I.lower_csc(M)


def _edge_cases():
    yield "n=1", *_spd_from_pattern(1, np.array([], int), np.array([], int), 0)
    yield "n=7 single ragged tile", *_spd_from_pattern(7, np.array([3, 6, 5]), np.array([0, 2, 1]), 1)
    yield "diagonal n=50", *_spd_from_pattern(50, np.array([], int), np.array([], int), 2)
    r, c = np.tril_indices(40, -1)
    yield "dense n=40", *_spd_from_pattern(40, r, c, 3)
    yield "tridiagonal n=64 (multiple of n_b)", *I.tridiag(64, 4)
    yield "arrowhead n=300, 6 dense rows last", *I.arrowhead(300, 6, 5)
    yield "disconnected blocks n=30", *_spd_from_pattern(30, np.array([1, 2, 20, 25]), np.array([0, 1, 18, 19]), 6)


EDGES = list(_edge_cases())


@pytest.mark.parametrize("route", ["semisparse", "dense", "supernodal"])
@pytest.mark.parametrize("nb", [8, 32])
@pytest.mark.parametrize("case", EDGES, ids=lambda c: c[0])
def test_edge_case_parity(case, nb, route):
    name, Ap, Ai, Ax = case
    n = len(Ap) - 1
    col = np.repeat(np.arange(n), np.diff(Ap))
    off = Ai != col
    rng = np.random.default_rng(n + nb)
    vals = np.stack([Ax, np.where(off, Ax * rng.uniform(-1, 1, len(Ax)), Ax)])
    P = Plan(n, Ap, Ai, nb=nb, route=route, ordering="natural")
    rhs = rng.standard_normal((2, 2, n))
    check_against_oracle(P, Ap, Ai, vals, rhs)


def _race_cases():
    n, bw = 5000, 200
    Ap, Ai = I.band_pattern(n, bw)
    vals = np.stack([I.band_values(n, bw, s, Ap, Ai) for s in range(4)])
    yield "band n=5000 bw 200, 2 slices", (n, Ap, Ai), dict(nb=128, ordering="natural", row_slices=2), vals
    yield "band n=5000 bw 200, 8 slices", (n, Ap, Ai), dict(nb=128, ordering="natural", row_slices=8), vals[:1]
    n2, bw2 = 3000, 40   # banded diagonal tiles whose later slices skip groups outside the band
    Ap2, Ai2 = I.band_pattern(n2, bw2)
    vals2 = np.stack([I.band_values(n2, bw2, s, Ap2, Ai2) for s in range(3)])
    yield "band n=3000 bw 40, 8 slices", (n2, Ap2, Ai2), dict(nb=128, ordering="natural", row_slices=8), vals2
    Ap, Ai, Ax, coords = I.laplace2d_bordered(seed=0)
    vals = np.stack([I.laplace2d_bordered(seed=s)[2] for s in range(3)])
    yield "config 1 (bordered 2-D), ND", (len(Ap) - 1, Ap, Ai), dict(coords=coords, nb=64), vals
    n = 517
    Ap, Ai, Ax = I.random_spd(n, 0.006, 1)
    col = np.repeat(np.arange(n), np.diff(Ap))
    vals = np.stack([Ax, np.where(Ai != col, -Ax, Ax)])
    yield "random indexed, n_b 16, RCM", (n, Ap, Ai), dict(nb=16, ordering="rcm", route="semisparse"), vals
    Ap, Ai, Ax, coords = I.fem3d(12, 11, 10)
    yield "3-D FEM, dense route", (len(Ap) - 1, Ap, Ai), dict(coords=coords, nb=32, route="dense", nd_leaf=32), Ax[None]


@pytest.mark.parametrize("case", list(_race_cases()), ids=lambda c: c[0])
def test_parallel_replay_matches_serial_bit_for_bit(case):
    name, (n, Ap, Ai), kw, vals = case
    batch = vals.shape[0]
    v = dev(vals)
    b = dev(np.random.default_rng(11).standard_normal((batch, 2, n)))
    out = {}
    for ctas in (1, 0, 3 * 152):
        P = Plan(n, Ap, Ai, replay_ctas=ctas, **kw)
        fac = P.factorize(v)
        assert fac.status() == L.STC_OK
        assert int(fac.info.abs().sum()) == 0
        ld = fac.logdet()
        x = fac.solve(b)
        sig = fac.selinv()
        assert sig.status() == L.STC_OK
        fac2, x2 = P.factorize_solve(v, b, check_status=True)
        out[ctas] = (fac.data.clone(), ld.clone(), x.clone(), sig.data.clone(), fac2.data.clone(), x2.clone())
    ref = out[1]
    for ctas in (0, 3 * 152):
        for what, a, r in zip(("factor", "logdet", "solve", "selected inverse", "fused factor", "fused solve"),
                              out[ctas], ref):
            assert torch.equal(a, r), "%s: %s differs from the serial replay (grid %d)" % (name, what, ctas)


@pytest.mark.parametrize("case", EDGES, ids=lambda c: c[0])
def test_edge_case_selected_inverse(case):
    # Sigma and d logdet / d a on the degenerate cases, both layouts
    from test_gpu_adjoint import _selinv_case
    name, Ap, Ai, Ax = case
    n = len(Ap) - 1
    for route in ("semisparse", "supernodal"):
        _selinv_case(Plan(n, Ap, Ai, nb=8, route=route, ordering="natural"), Ap, Ai, Ax[None])
