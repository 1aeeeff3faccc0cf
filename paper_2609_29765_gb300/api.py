"""Object API over the C ABI: analyze once, factorize many times (Sec. 6.6's split).

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

ROUTES = {"auto": L.STC_ROUTE_AUTO, "dense": L.STC_ROUTE_DENSE, "semisparse": L.STC_ROUTE_SEMISPARSE,
          "supernodal": L.STC_ROUTE_SUPERNODAL}
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
                 perm=None, nd_leaf=64, row_slices=0, spin_limit=0, replay_ctas=0, host_threads=0):
        o = L.stc_options_default()
        o.nb = int(nb)
        o.force_route = ROUTES[route]
        o.ordering = ORDERINGS[ordering if perm is None else "given"]
        o.nd_leaf = int(nd_leaf)
        o.row_slices = int(row_slices)
        o.spin_limit = int(spin_limit)
        o.replay_ctas = int(replay_ctas)
        o.host_threads = int(host_threads)
        self._perm_keep = None
        if perm is not None:
            self._perm_keep = np.ascontiguousarray(perm, dtype=np.int64)
            o.perm = self._perm_keep.ctypes.data_as(L.C.POINTER(L.C.c_int64))
        self.h = None
        rc, h = L.stc_analyze(n, colptr, rowind, coords, o)
        L.check(rc, "stc_analyze")
        self._adopt(h)

    def _adopt(self, h):
        self.h = h
        i = L.stc_plan_info_get(h)
        self.info = {f: getattr(i, f) for f, _ in L.stc_plan_info._fields_ if not f.startswith("reserved")}
        self.n, self.nnzA, self.nnzL = int(i.n), int(i.nnzA), int(i.nnzL)
        self._ws = {}

    def save(self) -> bytes:
        """The analysed plan as a self-contained blob (stc_plan_save)."""
        return L.stc_plan_save(self.h)

    @classmethod
    def load(cls, blob: bytes) -> "Plan":
        """A plan from a blob of `save`, without re-running the analysis (stc_plan_load)."""
        rc, h = L.stc_plan_load(bytes(blob))
        L.check(rc, "stc_plan_load")
        P = cls.__new__(cls)
        P._perm_keep = None
        P._adopt(h)
        return P

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
                "tile_offsets": L.STC_EXPORT_TILE_OFFSETS, "chunk_extents": L.STC_EXPORT_CHUNK_EXTENTS,
                "sn_nodes": L.STC_EXPORT_SN_NODES, "sn_rows": L.STC_EXPORT_SN_ROWS,
                "sn_cells": L.STC_EXPORT_SN_CELLS, "sn_tasks": L.STC_EXPORT_SN_TASKS,
                "sn_dev_cells": L.STC_EXPORT_SN_DEV_CELLS, "sn_dev_tasks": L.STC_EXPORT_SN_DEV_TASKS,
                "sn_dev_upds": L.STC_EXPORT_SN_DEV_UPDS, "sn_dev_maps": L.STC_EXPORT_SN_DEV_MAPS,
                "sn_value_map": L.STC_EXPORT_SN_VALUE_MAP, "sn_csc_map": L.STC_EXPORT_SN_CSC_MAP,
                "sn_sel_tasks": L.STC_EXPORT_SN_SEL_TASKS, "sn_sel_cons": L.STC_EXPORT_SN_SEL_CONS,
                "sn_cell_rowoff": L.STC_EXPORT_SN_CELL_ROWOFF}[what]
        a = L.stc_plan_export(self.h, code)
        if what == "tiles":
            return a.reshape(-1, 9)
        if what == "chunk_extents":
            return a.reshape(-1, 8, 2)
        if what in ("tasks", "sn_nodes", "sn_cells", "sn_tasks"):
            return a.reshape(-1, 4)
        if what in ("sn_dev_cells", "sn_dev_upds", "sn_sel_tasks"):
            return a.reshape(-1, 7)
        if what == "sn_sel_cons":
            return a.reshape(-1, 3)
        if what == "sn_dev_tasks":
            return a.reshape(-1, 8)
        return a

    def factor_bytes(self, batch: int = 1) -> int:
        return L.stc_factor_bytes(self.h, batch)

    def workspace_bytes(self, batch: int = 1) -> int:
        return L.stc_workspace_bytes(self.h, batch)

    def upload(self):
        L.check(L.stc_plan_upload(self.h), "stc_plan_upload")

    def workspace(self, batch: int, device=None, nbytes=None):
        torch = _torch()
        nbytes = self.workspace_bytes(batch) if nbytes is None else max(int(nbytes), self.workspace_bytes(batch))
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


    def factorize_solve(self, values, b, check_status=False):
        """Factorize and solve in one call (the value upload and the forward substitution
        run inside the factorization's launch): values [batch, nnzA], b [batch, nrhs, n]
        (or [batch, n]), float64 on the GPU or in pinned host memory (read by the kernels
        in place, where the platform maps pinned host memory for the device, as over
        NVLink-C2C).  Returns (Factor, x) with x on the GPU; the factor is the one
        factorize() gives."""
        torch = _torch()
        if values.dim() == 1:
            values = values.unsqueeze(0)
        if values.dtype != torch.float64 or values.shape[1] != self.nnzA:
            raise ValueError("values must be float64 [batch, nnzA=%d]" % self.nnzA)
        values = values.contiguous()
        batch = values.shape[0]
        squeeze = b.dim() == 2
        if squeeze:
            b = b.unsqueeze(1)
        b = b.contiguous()
        if b.shape[0] != batch or b.shape[2] != self.n or b.dtype != torch.float64:
            raise ValueError("b must be float64 [batch, nrhs, n]")
        nrhs = b.shape[1]
        # values and b may be pinned host tensors: the kernels then read them in place
        dev = values.device if values.is_cuda else torch.device("cuda", torch.cuda.current_device())
        fac = torch.empty(self.factor_bytes(batch) // 8, dtype=torch.float64, device=dev)
        info = torch.empty(batch, dtype=torch.int32, device=dev)
        x = torch.empty(b.shape, dtype=torch.float64, device=dev)
        ws = self.workspace(batch, dev, L.stc_factorize_solve_workspace_bytes(self.h, batch, nrhs))
        L.check(L.stc_factorize_solve(self.h, values, batch, nrhs, b, fac, x, ws, info), "stc_factorize_solve")
        if check_status:
            L.check(L.stc_sync_status(ws), "stc_factorize_solve (device status)")
        return Factor(self, fac, info, batch), (x.squeeze(1) if squeeze else x)


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

    def selinv(self, out=None):
        """Selected inverse in tile storage (same layout as the factor)."""
        torch = _torch()
        sig = torch.empty_like(self.data) if out is None else out
        ws = self.plan.workspace(self.batch, self.data.device)
        L.check(L.stc_selinv(self.plan.h, self.data, self.batch, sig, ws), "stc_selinv")
        return Factor(self.plan, sig, self.info, self.batch)

    def logdet_backward(self, gout=None, out=None, accumulate=False):
        """(2 - delta_ij) (A^{-1})_ij * gout for every stored A entry: [batch, nnzA]."""
        torch = _torch()
        g = torch.empty(self.batch, self.plan.nnzA, dtype=torch.float64, device=self.data.device) \
            if out is None else out
        sig = torch.empty_like(self.data)
        ws = self.plan.workspace(self.batch, self.data.device)
        if gout is not None:
            gout = gout.to(dtype=torch.float64).contiguous()
        L.check(L.stc_logdet_backward(self.plan.h, self.data, self.batch, gout, g, int(accumulate), sig, ws),
                "stc_logdet_backward")
        return g

    def to_csc(self):
        """L's values in the CSC order of plan.export('Lp'/'Li'): [batch, nnzL]."""
        torch = _torch()
        out = torch.empty(self.batch, self.plan.nnzL, dtype=torch.float64, device=self.data.device)
        L.check(L.stc_factor_to_csc(self.plan.h, self.data, self.batch, out), "stc_factor_to_csc")
        return out


class GraphedFactorize:
    """scatter + factorize + logdet of a fixed batch size captured in one CUDA graph.

    First use of a plan on a device uploads its metadata (synchronous); that happens in
    a warm-up run before capture, after which every library call on the stream is a
    kernel launch or a memset, so the whole step replays as one graph launch.
    """

    def __init__(self, plan: Plan, batch: int, device=None):
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.plan, self.batch = plan, int(batch)
        plan.upload()
        self.values = torch.zeros(self.batch, plan.nnzA, dtype=torch.float64, device=dev)
        self.factor = torch.empty(plan.factor_bytes(self.batch) // 8, dtype=torch.float64, device=dev)
        self.info = torch.empty(self.batch, dtype=torch.int32, device=dev)
        self.logdet = torch.empty(self.batch, dtype=torch.float64, device=dev)
        self.ws = plan.workspace(self.batch, dev)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self._step()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._step()

    def _step(self):
        L.check(L.stc_factorize(self.plan.h, self.values, self.batch, self.factor, self.ws, self.info),
                "stc_factorize")
        L.check(L.stc_logdet(self.plan.h, self.factor, self.batch, self.logdet), "stc_logdet")

    def __call__(self, values):
        """Copy values [batch, nnzA] into the graph's input and replay; returns logdet."""
        self.values.copy_(values)
        self.graph.replay()
        return self.logdet

    def factor_view(self) -> "Factor":
        return Factor(self.plan, self.factor, self.info, self.batch)


class Group:
    """Several plans, each with its own batch, factorized by one persistent launch."""

    def __init__(self, plans, batches):
        self.plans, self.batches = list(plans), [int(b) for b in batches]
        self.h = None
        rc, h = L.stc_group_create([p.h for p in self.plans], self.batches)
        L.check(rc, "stc_group_create")
        self.h = h
        self._ws = None

    def __del__(self):
        if getattr(self, "h", None):
            L.stc_group_destroy(self.h)
            self.h = None

    def factorize(self, values_list):
        """values_list[p]: CUDA float64 [batch_p, nnzA_p]; returns one Factor per plan."""
        torch = _torch()
        dev = values_list[0].device
        facs, infos = [], []
        for P, b, v in zip(self.plans, self.batches, values_list):
            if v.shape != (b, P.nnzA) or v.dtype != torch.float64:
                raise ValueError("values must be float64 [batch_p, nnzA_p]")
            facs.append(torch.empty(P.factor_bytes(b) // 8, dtype=torch.float64, device=dev))
            infos.append(torch.empty(b, dtype=torch.int32, device=dev))
        nbytes = L.stc_group_workspace_bytes(self.h)
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 64), dtype=torch.uint8, device=dev)
        vals = [v.contiguous() for v in values_list]
        L.check(L.stc_factorize_group(self.h, vals, facs, infos, self._ws), "stc_factorize_group")
        return [Factor(P, f, i, b) for P, f, i, b in zip(self.plans, facs, infos, self.batches)]

    def status(self) -> int:
        return L.stc_sync_status(self._ws)


def factorize_mixed(plans, values_list):
    """Several patterns in one launch and one call (stc_factorize_mixed, synchronous):
    values_list[p] is CUDA float64 [batch_p, nnzA_p]; returns one Factor per plan."""
    torch = _torch()
    dev = values_list[0].device
    facs, infos, vals = [], [], []
    for P, v in zip(plans, values_list):
        if v.dim() != 2 or v.shape[1] != P.nnzA or v.dtype != torch.float64:
            raise ValueError("values must be float64 [batch_p, nnzA_p]")
        vals.append(v.contiguous())
        facs.append(torch.empty(P.factor_bytes(v.shape[0]) // 8, dtype=torch.float64, device=dev))
        infos.append(torch.empty(v.shape[0], dtype=torch.int32, device=dev))
    L.check(L.stc_factorize_mixed([P.h for P in plans], vals, [v.shape[0] for v in vals], facs, infos),
            "stc_factorize_mixed")
    return [Factor(P, f, i, v.shape[0]) for P, f, i, v in zip(plans, facs, infos, vals)]


# ---------------------------------------------------------------------------
# Differentiation: torch.autograd.Function wrappers.  The forward and backward
# arithmetic runs in libstc.so; torch only carries the tensors and the chain rule of
# whatever produced the values (e.g. Q(theta)).
# ---------------------------------------------------------------------------
def _autograd():
    torch = _torch()

    class LogdetFn(torch.autograd.Function):
        """logdet(A_b) for values [batch, nnzA]; backward = selected inverse."""

        @staticmethod
        def forward(ctx, values, plan):
            fac = plan.factorize(values.detach())
            ctx.plan, ctx.fac = plan, fac
            return fac.logdet()

        @staticmethod
        def backward(ctx, gout):
            g = ctx.fac.logdet_backward(gout.contiguous())
            return g, None

    class QuadFn(torch.autograd.Function):
        """x_b^T A_b x_b; gradients for the values and for x."""

        @staticmethod
        def forward(ctx, values, x, plan):
            values = values.detach().contiguous()
            x = x.detach().contiguous()
            out = torch.empty(values.shape[0], dtype=torch.float64, device=values.device)
            L.check(L.stc_quad_form(plan.h, values.shape[0], values, x, out), "stc_quad_form")
            ctx.save_for_backward(values, x)
            ctx.plan = plan
            return out

        @staticmethod
        def backward(ctx, gout):
            values, x = ctx.saved_tensors
            plan = ctx.plan
            batch = values.shape[0]
            gv = gx = None
            if ctx.needs_input_grad[0]:
                gv = torch.empty_like(values)
                L.check(L.stc_sym_outer_backward(plan.h, batch, x, x, gout.contiguous(), gv, 0),
                        "stc_sym_outer_backward")
            if ctx.needs_input_grad[1]:
                raise RuntimeError("quad_form: the gradient with respect to x is not provided "
                                   "(treat x as a constant, or use solve for x-dependent terms)")
            return gv, gx, None

    class SolveFn(torch.autograd.Function):
        """x = A_b^{-1} b_b; backward: g_b = A^{-1} g_x, g_A = -(2-delta)/2 (x_i g_j + x_j g_i)."""

        @staticmethod
        def forward(ctx, values, b, plan):
            fac = plan.factorize(values.detach())
            x = fac.solve(b.detach().contiguous())
            ctx.plan, ctx.fac = plan, fac
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            g = ctx.fac.solve(gx.contiguous())
            gv = None
            if ctx.needs_input_grad[0]:
                batch = x.shape[0]
                gv = torch.empty(batch, ctx.plan.nnzA, dtype=torch.float64, device=x.device)
                scale = torch.full((batch,), -1.0, dtype=torch.float64, device=x.device)
                L.check(L.stc_sym_outer_backward(ctx.plan.h, batch, x.contiguous(), g.contiguous(), scale, gv, 0),
                        "stc_sym_outer_backward")
            return gv, g, None

    return LogdetFn, QuadFn, SolveFn


def logdet(values, plan):
    """Differentiable logdet of each value set: values [batch, nnzA] -> [batch]."""
    return _autograd()[0].apply(values, plan)


def quad_form(values, x, plan):
    """Differentiable x_b^T A_b x_b."""
    return _autograd()[1].apply(values, x, plan)


def solve(values, b, plan):
    """Differentiable x = A^{-1} b, b [batch, n]."""
    return _autograd()[2].apply(values, b, plan)
