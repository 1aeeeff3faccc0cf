"""Object API over the C ABI: analyze once, factorize many times (Sec. 6.7's split).

    plan = Plan(n, Ap, Ai, coords=coords, nb=64)        # host analysis
    fac = plan.factorize(values)                          # values: CUDA float64 [batch, nnzA]
    ld = fac.logdet()                                     # CUDA float64 [batch]
    x = fac.solve(b)                                      # b: CUDA float64 [batch, nrhs, n]

PyTorch provides device memory and the current stream; every step of the numeric path
runs in libstc.so's kernels.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L

ROUTES = {"auto": L.STC_ROUTE_AUTO, "dense": L.STC_ROUTE_DENSE, "semisparse": L.STC_ROUTE_SEMISPARSE}
ROUTE_NAMES = {L.STC_ROUTE_DENSE: "dense", L.STC_ROUTE_SEMISPARSE: "semisparse",
               L.STC_ROUTE_SUPERNODAL: "supernodal"}
ORDERINGS = {"auto": L.STC_ORDER_AUTO, "natural": L.STC_ORDER_NATURAL, "given": L.STC_ORDER_GIVEN,
             "nd": L.STC_ORDER_ND, "rcm": L.STC_ORDER_RCM}


def _torch():
    import torch
    return torch


class Plan:
    """Symbolic plan of one sparsity pattern (lower CSC, original order)."""

    def __init__(self, n, colptr, rowind, coords=None, nb=128, route="auto", ordering="auto",
                 perm=None, nd_leaf=64, row_slices=0, spin_limit=0):
        o = L.stc_options_default()
        o.nb = int(nb)
        o.force_route = ROUTES[route]
        o.ordering = ORDERINGS[ordering if perm is None else "given"]
        o.nd_leaf = int(nd_leaf)
        o.row_slices = int(row_slices)
        o.spin_limit = int(spin_limit)
        self._perm_keep = None
        if perm is not None:
            self._perm_keep = np.ascontiguousarray(perm, dtype=np.int64)
            o.perm = self._perm_keep.ctypes.data_as(L.C.POINTER(L.C.c_int64))
        self.h = None
        rc, h = L.stc_analyze(n, colptr, rowind, coords, o)
        L.check(rc, "stc_analyze")
        self.h = h
        i = L.stc_plan_info_get(h)
        self.info = {f: getattr(i, f) for f, _ in L.stc_plan_info._fields_ if not f.startswith("reserved")}
        self.n, self.nnzA, self.nnzL = int(i.n), int(i.nnzA), int(i.nnzL)
        self._ws = {}

    def __del__(self):
        if getattr(self, "h", None):
            L.stc_plan_destroy(self.h)
            self.h = None

    @property
    def route(self) -> str:
        return ROUTE_NAMES[self.info["route_executed"]]

    @property
    def route_selected(self) -> str:
        return ROUTE_NAMES[self.info["route_selected"]]

    def export(self, what: str) -> np.ndarray:
        code = {"perm": L.STC_EXPORT_PERM, "etree": L.STC_EXPORT_ETREE, "Lp": L.STC_EXPORT_LP,
                "Li": L.STC_EXPORT_LI, "tiles": L.STC_EXPORT_TILES, "aind": L.STC_EXPORT_AIND,
                "tasks": L.STC_EXPORT_TASKS, "value_map": L.STC_EXPORT_VALUE_MAP,
                "tile_offsets": L.STC_EXPORT_TILE_OFFSETS}[what]
        a = L.stc_plan_export(self.h, code)
        if what == "tiles":
            return a.reshape(-1, 9)
        if what == "tasks":
            return a.reshape(-1, 4)
        return a

    def factor_bytes(self, batch: int = 1) -> int:
        return L.stc_factor_bytes(self.h, batch)

    def workspace_bytes(self, batch: int = 1) -> int:
        return L.stc_workspace_bytes(self.h, batch)

    def upload(self):
        L.check(L.stc_plan_upload(self.h), "stc_plan_upload")

    def workspace(self, batch: int, device=None):
        torch = _torch()
        nbytes = self.workspace_bytes(batch)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        w = self._ws.get(dev)
        if w is None or w.numel() < nbytes:
            w = torch.empty(max(nbytes, 64), dtype=torch.uint8, device=dev)
            self._ws[dev] = w
        return w

    def factorize(self, values, out=None, check_status=False) -> "Factor":
        """values: CUDA float64 [batch, nnzA] (or [nnzA]) in the pattern's CSC order."""
        torch = _torch()
        if values.dim() == 1:
            values = values.unsqueeze(0)
        if values.dtype != torch.float64 or values.shape[1] != self.nnzA:
            raise ValueError("values must be float64 [batch, nnzA=%d]" % self.nnzA)
        values = values.contiguous()
        batch = values.shape[0]
        if out is None:
            fac = torch.empty(self.factor_bytes(batch) // 8, dtype=torch.float64, device=values.device)
            info = torch.empty(batch, dtype=torch.int32, device=values.device)
        else:
            fac, info = out
        ws = self.workspace(batch, values.device)
        L.check(L.stc_factorize(self.h, values, batch, fac, ws, info), "stc_factorize")
        if check_status:
            L.check(L.stc_sync_status(ws), "stc_factorize (device status)")
        return Factor(self, fac, info, batch)


class Factor:
    """A batch of factors in tile storage on the device."""

    def __init__(self, plan: Plan, data, info, batch: int):
        self.plan, self.data, self.info, self.batch = plan, data, info, int(batch)

    def status(self) -> int:
        return L.stc_sync_status(self.plan.workspace(self.batch, self.data.device))

    def logdet(self, out=None):
        torch = _torch()
        out = torch.empty(self.batch, dtype=torch.float64, device=self.data.device) if out is None else out
        L.check(L.stc_logdet(self.plan.h, self.data, self.batch, out), "stc_logdet")
        return out

    def solve(self, b, out=None):
        """b: CUDA float64 [batch, nrhs, n] (or [batch, n]); returns x of the same shape."""
        torch = _torch()
        squeeze = b.dim() == 2
        if squeeze:
            b = b.unsqueeze(1)
        b = b.contiguous()
        if b.shape[0] != self.batch or b.shape[2] != self.plan.n or b.dtype != torch.float64:
            raise ValueError("b must be float64 [batch, nrhs, n]")
        nrhs = b.shape[1]
        x = torch.empty_like(b) if out is None else out
        ws = self.plan.workspace(self.batch * nrhs, b.device)
        L.check(L.stc_solve(self.plan.h, self.data, self.batch, nrhs, b, x, ws), "stc_solve")
        return x.squeeze(1) if squeeze else x

    def to_csc(self):
        """L's values in the CSC order of plan.export('Lp'/'Li'): [batch, nnzL]."""
        torch = _torch()
        out = torch.empty(self.batch, self.plan.nnzL, dtype=torch.float64, device=self.data.device)
        L.check(L.stc_factor_to_csc(self.plan.h, self.data, self.batch, out), "stc_factor_to_csc")
        return out
