"""Batching forms: mixed patterns in one launch, CUDA-graph replay, the autotuner."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import GraphedFactorize, Group, Plan, factorize_mixed
from paper_2609_29765_gb300.tune import autotune

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("route", ["dense", "semisparse", "supernodal", "mixed"])
def test_group_mixed_patterns_match_single_launch_and_oracle(route):
    # "mixed": one plan per route in the same launch (the kernel that also runs
    # supernodal tasks)
    plans, vals, pats = [], [], []
    for i, (m, b) in enumerate(((8, 2), (10, 3), (12, 2))):   # 8^3, 10^3, 12^3 grids, uneven batches
        vs = []
        for s in range(b):
            Ap, Ai, Ax, coords = I.fem3d(m, m, m, seed=s)
            vs.append(Ax)
        pats.append((len(Ap) - 1, Ap, Ai))
        r = ("dense", "supernodal", "semisparse")[i] if route == "mixed" else route
        plans.append(Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=32, route=r, nd_leaf=32))
        vals.append(dev(np.stack(vs)))
    G = Group(plans, [v.shape[0] for v in vals])
    facs = G.factorize(vals)
    assert G.status() == L.STC_OK
    once = factorize_mixed(plans, vals)                   # the one-call form
    for P, v, f, g, (n, Ap, Ai) in zip(plans, vals, facs, once, pats):
        ref = P.factorize(v)
        assert torch.equal(f.to_csc(), ref.to_csc())     # same tasks, same arithmetic
        assert torch.equal(g.to_csc(), ref.to_csc())
        assert int(f.info.abs().sum()) == 0
        F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
        Lo, _ = F.factor(v[-1].cpu().numpy())
        ld = f.logdet().cpu().numpy()[-1]
        assert abs(ld - F.logdet(Lo)) <= 1e-10 * abs(F.logdet(Lo))


def test_cuda_graph_replay_matches_direct_calls():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64)
    g = GraphedFactorize(P, 4)
    for seeds in ([0, 1, 2, 3], [4, 5, 6, 7]):
        v = dev(np.stack([I.laplace2d_bordered(seed=s)[2] for s in seeds]))
        ld = g(v).clone()
        ref = P.factorize(v).logdet()
        assert torch.equal(ld, ref)
        assert torch.equal(g.factor_view().to_csc(), P.factorize(v).to_csc())


def test_autotuner_picks_a_valid_configuration():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    n = len(Ap) - 1
    v = dev(np.stack([I.laplace2d_bordered(seed=s)[2] for s in range(8)]))
    best, table = autotune(n, Ap, Ai, v, coords=coords, nbs=(32, 64), slices=(1, 2), reps=1)
    assert len(table) == 9 and all(r["ok"] for r in table)   # 2 tile routes x 4, supernodal once
    assert {r["route"] for r in table} == {"semisparse", "dense", "supernodal"}
    assert best["ms"] == min(r["ms"] for r in table)
    P = Plan(n, Ap, Ai, coords=coords, nb=best["nb"], row_slices=best["row_slices"], route=best["route"])
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    Lo, _ = F.factor(v[3].cpu().numpy())
    ld = P.factorize(v).logdet().cpu().numpy()[3]
    assert abs(ld - F.logdet(Lo)) <= 1e-10 * abs(F.logdet(Lo))
