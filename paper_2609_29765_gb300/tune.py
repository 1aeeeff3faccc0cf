"""Autotuner: pick the route, the tile size n_b and the row-slice count for a pattern and batch.

Grid search, measured on the device: for every candidate n_b the pattern is analysed on
the host (ordering and symbolic factor are shared by construction of the inputs), and
for every row-slice count the factorization of the caller's values is timed with CUDA
events (best of `reps` after one warm-up).  The row-slice count is how many device tasks
an off-diagonal tile's rows (and a diagonal tile's SYRK rows) are split into -- the
height of the active-column panel one CTA owns.  Returns the fastest configuration and
the full table.
"""
from __future__ import annotations

from . import _lib as L
from .api import Plan


def autotune(n, colptr, rowind, values, coords=None, nbs=(32, 64, 96, 128), slices=(1, 2, 4, 8),
             route="auto", ordering="auto", reps=2, nd_leaf=64):
    """route="auto" also tries the three routes (the supernodal layout once: n_b and the
    row slices do not change it); a named route tunes n_b and the slices of that route."""
    import torch
    if values.dim() == 1:
        values = values.unsqueeze(0)
    values = values.contiguous()
    batch = values.shape[0]
    table = []
    configs = []
    for r in (("semisparse", "dense", "supernodal") if route == "auto" else (route,)):
        if r == "supernodal":
            configs.append((r, nbs[0], slices[0]))
        else:
            configs += [(r, nb, s) for nb in nbs for s in slices]
    for r, nb, s in configs:
        if True:
            P = Plan(n, colptr, rowind, coords=coords, nb=nb, route=r, ordering=ordering,
                     row_slices=s, nd_leaf=nd_leaf)
            fac = torch.empty(P.factor_bytes(batch) // 8, dtype=torch.float64, device=values.device)
            info = torch.empty(batch, dtype=torch.int32, device=values.device)
            ws = P.workspace(batch, values.device)
            L.check(L.stc_factorize(P.h, values, batch, fac, ws, info), "stc_factorize")
            L.check(L.stc_sync_status(ws), "autotune warm-up")
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                L.check(L.stc_factorize(P.h, values, batch, fac, ws, info), "stc_factorize")
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            ok = int(info.abs().sum().item()) == 0
            table.append({"nb": nb, "row_slices": s, "ms": best, "ok": ok,
                          "route": P.route, "flops_tile": P.info["flops_tile"]})
            del fac, info
    good = [r for r in table if r["ok"]]
    best = min(good or table, key=lambda r: r["ms"])
    return best, table
