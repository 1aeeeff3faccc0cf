"""Randomized GPU parity: random patterns, tile sizes, orderings, routes and batch sizes,
factorize / logdet / solve against the oracle with the tolerances of test_gpu_factor.py.

Values of the extra items keep the first item's diagonal and scale its off-diagonal
entries by U(-1, 1), so every item stays diagonally dominant (SPD).
"""
import numpy as np
import pytest

from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan
from test_gpu_factor import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(10))
def test_random_pattern_parity(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(30, 420))
    Ap, Ai, Ax = I.random_spd(n, float(rng.uniform(0.004, 0.06)), 700 + seed)
    nb = int(rng.choice([8, 16, 32, 48, 64, 128]))
    route = "dense" if seed % 3 == 0 else "semisparse"
    ordering = ["rcm", "natural", "given"][seed % 3]
    perm = rng.permutation(n) if ordering == "given" else None
    batch = int(rng.integers(1, 4))
    col = np.repeat(np.arange(n), np.diff(Ap))
    off = Ai != col
    vals = np.stack([Ax] + [np.where(off, Ax * rng.uniform(-1, 1, len(Ax)), Ax) for _ in range(batch - 1)])
    P = Plan(n, Ap, Ai, nb=nb, route=route, ordering=ordering if perm is None else "auto", perm=perm,
             row_slices=int(rng.choice([0, 1, 2, 4, 8])))
    rhs = rng.standard_normal((batch, 2, n))
    check_against_oracle(P, Ap, Ai, vals, rhs)
