"""ctypes binding of libstc.so (include/stc.h).  Argument marshalling only.

Every function carries the C name and takes numpy arrays (host) or torch CUDA tensors
(device); it converts them to pointers and returns the C status code.  The library is
loaded from the package's _build directory; if it is not there this module raises at
import time of the first call: there is no CPU fallback anywhere in the product.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

STC_OK = 0
STC_ERR_INVALID_ARG = -1
STC_ERR_INVALID_PATTERN = -2
STC_ERR_OUT_OF_MEMORY = -3
STC_ERR_CUDA = -4
STC_ERR_TIMEOUT = -5
STC_ERR_UNSUPPORTED = -6
STC_ERR_BUFFER_TOO_SMALL = -7

STC_ROUTE_AUTO, STC_ROUTE_DENSE, STC_ROUTE_SEMISPARSE, STC_ROUTE_SUPERNODAL = -1, 0, 1, 2
STC_ORDER_AUTO, STC_ORDER_NATURAL, STC_ORDER_GIVEN, STC_ORDER_ND, STC_ORDER_RCM = 0, 1, 2, 3, 4
(STC_EXPORT_PERM, STC_EXPORT_ETREE, STC_EXPORT_LP, STC_EXPORT_LI, STC_EXPORT_TILES, STC_EXPORT_AIND,
 STC_EXPORT_TASKS, STC_EXPORT_VALUE_MAP, STC_EXPORT_TILE_OFFSETS, STC_EXPORT_CHUNK_EXTENTS,
 STC_EXPORT_SN_NODES, STC_EXPORT_SN_ROWS, STC_EXPORT_SN_CELLS, STC_EXPORT_SN_TASKS,
 STC_EXPORT_SN_DEV_CELLS, STC_EXPORT_SN_DEV_TASKS, STC_EXPORT_SN_DEV_UPDS, STC_EXPORT_SN_DEV_MAPS,
 STC_EXPORT_SN_VALUE_MAP, STC_EXPORT_SN_CSC_MAP, STC_EXPORT_SN_SEL_TASKS, STC_EXPORT_SN_SEL_CONS,
 STC_EXPORT_SN_CELL_ROWOFF) = range(23)

# every symbol include/stc.h declares
EXPORTED = [
    "stc_options_default", "stc_analyze", "stc_plan_info_get", "stc_plan_export", "stc_plan_upload",
    "stc_plan_destroy", "stc_factor_bytes", "stc_workspace_bytes", "stc_factorize", "stc_scatter_values",
    "stc_factorize_scattered", "stc_sync_status",
    "stc_logdet", "stc_solve", "stc_factor_to_csc", "stc_fp64_peak_probe", "stc_factorize_noalloc",
    "stc_selinv", "stc_logdet_backward", "stc_sym_outer_backward", "stc_quad_form",
    "stc_group_create", "stc_group_workspace_bytes", "stc_factorize_group", "stc_group_destroy",
    "stc_strerror", "stc_factorize_mixed", "stc_quad_backward", "stc_plan_save", "stc_plan_load",
    "stc_plan_export_taskset", "stc_plan_sync_status", "stc_factorize_solve",
    "stc_factorize_solve_workspace_bytes", "stc_factorize_forward", "stc_solve_backward",
    "stc_factorize_forward_fills",
]
(STC_TASKSET_TASKS, STC_TASKSET_UPDS, STC_TASKSET_IMAP, STC_TASKSET_TILES, STC_TASKSET_SAIND,
 STC_TASKSET_CEXT, STC_TASKSET_CSC_MAP, STC_TASKSET_PAD_DIAG) = range(8)
STC_NOALLOC_SCRATCH_BYTES = 4 << 20


def stc_strerror(code) -> str:
    return lib().stc_strerror(int(code)).decode()


class StcError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__("%s: %s (%d)" % (where, stc_strerror(code), code))
        self.code = code


class stc_options(C.Structure):
    _fields_ = [("nb", C.c_int32), ("force_route", C.c_int32), ("ordering", C.c_int32),
                ("nd_leaf", C.c_int32), ("perm", C.POINTER(C.c_int64)), ("row_slices", C.c_int32),
                ("host_threads", C.c_int32), ("spin_limit", C.c_int64), ("gate_rho_dense", C.c_double),
                ("gate_phi_fill", C.c_double), ("gate_rho_semi", C.c_double),
                ("gate_sigma_skew", C.c_double), ("replay_ctas", C.c_int32), ("reserved1", C.c_int32)]


class stc_plan_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nb", C.c_int64), ("nt", C.c_int64), ("ntiles", C.c_int64),
                ("nnzA", C.c_int64), ("nnzL", C.c_int64), ("stored_entries", C.c_int64),
                ("factor_doubles", C.c_int64), ("route_selected", C.c_int32),
                ("route_executed", C.c_int32), ("ordering", C.c_int32), ("reserved0", C.c_int32),
                ("phi", C.c_double), ("rho", C.c_double), ("sigma", C.c_double),
                ("ntasks_alg1", C.c_int64), ("n_potrf", C.c_int64), ("n_syrk", C.c_int64),
                ("n_trsm", C.c_int64), ("n_gemm", C.c_int64), ("flops_alg", C.c_double),
                ("flops_tile", C.c_double), ("analyze_seconds", C.c_double)]


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def lib():
    """Load libstc.so (building it first only when it has never been built here)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            _build.build()
        L = C.CDLL(_build.LIB)
        L.stc_options_default.argtypes = [C.POINTER(stc_options)]
        L.stc_options_default.restype = None
        L.stc_strerror.argtypes = [C.c_int]
        L.stc_strerror.restype = C.c_char_p
        L.stc_analyze.argtypes = [C.c_int64, _vp, _vp, _vp, C.POINTER(stc_options), C.POINTER(_vp)]
        L.stc_analyze.restype = C.c_int
        L.stc_plan_info_get.argtypes = [_vp, C.POINTER(stc_plan_info)]
        L.stc_plan_info_get.restype = C.c_int
        L.stc_plan_export.argtypes = [_vp, C.c_int, _vp, C.POINTER(C.c_size_t)]
        L.stc_plan_export.restype = C.c_int
        L.stc_plan_upload.argtypes = [_vp]
        L.stc_plan_upload.restype = C.c_int
        L.stc_plan_destroy.argtypes = [_vp]
        L.stc_plan_destroy.restype = None
        L.stc_plan_export_taskset.argtypes = [_vp, C.c_int32, C.c_int, C.c_int, _vp, C.POINTER(C.c_size_t)]
        L.stc_plan_export_taskset.restype = C.c_int
        L.stc_plan_save.argtypes = [_vp, _vp, C.POINTER(C.c_size_t)]
        L.stc_plan_save.restype = C.c_int
        L.stc_plan_load.argtypes = [_vp, C.c_size_t, C.POINTER(_vp)]
        L.stc_plan_load.restype = C.c_int
        L.stc_factor_bytes.argtypes = [_vp, C.c_int64]
        L.stc_factor_bytes.restype = C.c_size_t
        L.stc_workspace_bytes.argtypes = [_vp, C.c_int64]
        L.stc_workspace_bytes.restype = C.c_size_t
        L.stc_factorize.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]
        L.stc_factorize.restype = C.c_int
        L.stc_scatter_values.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.stc_scatter_values.restype = C.c_int
        L.stc_factorize_scattered.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, _vp]
        L.stc_factorize_scattered.restype = C.c_int
        L.stc_sync_status.argtypes = [_vp, _vp]
        L.stc_sync_status.restype = C.c_int
        L.stc_plan_sync_status.argtypes = [_vp, _vp]
        L.stc_plan_sync_status.restype = C.c_int
        L.stc_logdet.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.stc_logdet.restype = C.c_int
        L.stc_solve.argtypes = [_vp, _vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp]
        L.stc_solve.restype = C.c_int
        L.stc_factorize_solve.argtypes = [_vp, _vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
        L.stc_factorize_solve.restype = C.c_int
        L.stc_factorize_solve_workspace_bytes.argtypes = [_vp, C.c_int64, C.c_int64]
        L.stc_factorize_solve_workspace_bytes.restype = C.c_size_t
        L.stc_factorize_forward.argtypes = [_vp, _vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp]
        L.stc_factorize_forward.restype = C.c_int
        L.stc_solve_backward.argtypes = [_vp, _vp, C.c_int64, C.c_int64, _vp, _vp, _vp]
        L.stc_solve_backward.restype = C.c_int
        L.stc_factorize_forward_fills.argtypes = [_vp, C.c_int64]
        L.stc_factorize_forward_fills.restype = C.c_int
        L.stc_factor_to_csc.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.stc_factor_to_csc.restype = C.c_int
        L.stc_group_create.argtypes = [C.c_int32, C.POINTER(_vp), C.POINTER(C.c_int64), C.POINTER(_vp)]
        L.stc_group_create.restype = C.c_int
        L.stc_group_workspace_bytes.argtypes = [_vp]
        L.stc_group_workspace_bytes.restype = C.c_size_t
        L.stc_factorize_group.argtypes = [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _vp, _vp]
        L.stc_factorize_group.restype = C.c_int
        L.stc_factorize_mixed.argtypes = [C.c_int32, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_int64),
                                          C.POINTER(_vp), C.POINTER(_vp), _vp]
        L.stc_factorize_mixed.restype = C.c_int
        L.stc_quad_backward.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, C.c_int, _vp]
        L.stc_quad_backward.restype = C.c_int
        L.stc_group_destroy.argtypes = [_vp]
        L.stc_group_destroy.restype = None
        L.stc_selinv.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp]
        L.stc_selinv.restype = C.c_int
        L.stc_logdet_backward.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, C.c_int, _vp, _vp, _vp]
        L.stc_logdet_backward.restype = C.c_int
        L.stc_sym_outer_backward.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, _vp, C.c_int, _vp]
        L.stc_sym_outer_backward.restype = C.c_int
        L.stc_quad_form.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, _vp]
        L.stc_quad_form.restype = C.c_int
        L.stc_factorize_noalloc.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]
        L.stc_factorize_noalloc.restype = C.c_int
        L.stc_fp64_peak_probe.argtypes = [_vp, C.c_int64, C.c_int64, C.POINTER(C.c_double)]
        L.stc_fp64_peak_probe.restype = C.c_int
        _lib = L
        return L


def check(code, where=""):
    if code != STC_OK:
        raise StcError(code, where)
    return code


def _host_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _in_ptr(t):
    """An input the kernels read: a CUDA tensor, or a pinned host tensor (read by the
    kernels in place where the platform maps pinned host memory for the device)."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError("expected a CUDA tensor or a pinned host tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return C.c_void_p(t.data_ptr())
    return _dev_ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---- C-named marshalling wrappers ------------------------------------------------
def stc_options_default() -> stc_options:
    o = stc_options()
    lib().stc_options_default(C.byref(o))
    return o


def stc_analyze(n, colptr, rowind, coords=None, opt: stc_options | None = None):
    """Returns (status, plan_handle)."""
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int64)
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64)
    h = C.c_void_p()
    rc = lib().stc_analyze(int(n), _host_ptr(colptr), _host_ptr(rowind), _host_ptr(coords),
                           C.byref(opt) if opt is not None else None, C.byref(h))
    return rc, h


def stc_plan_info_get(plan) -> stc_plan_info:
    info = stc_plan_info()
    check(lib().stc_plan_info_get(plan, C.byref(info)), "stc_plan_info_get")
    return info


def stc_plan_export(plan, what: int) -> np.ndarray:
    sz = C.c_size_t(0)
    check(lib().stc_plan_export(plan, int(what), None, C.byref(sz)), "stc_plan_export")
    out = np.empty(sz.value // 8, dtype=np.int64)
    check(lib().stc_plan_export(plan, int(what), _host_ptr(out), C.byref(sz)), "stc_plan_export")
    return out


def stc_plan_export_taskset(plan, slices: int, bl_order: bool, what: int) -> np.ndarray:
    sz = C.c_size_t(0)
    check(lib().stc_plan_export_taskset(plan, int(slices), int(bl_order), int(what), None, C.byref(sz)),
          "stc_plan_export_taskset")
    out = np.empty(sz.value // 8, dtype=np.int64)
    check(lib().stc_plan_export_taskset(plan, int(slices), int(bl_order), int(what), _host_ptr(out), C.byref(sz)),
          "stc_plan_export_taskset")
    return out


def stc_plan_save(plan) -> bytes:
    sz = C.c_size_t(0)
    check(lib().stc_plan_save(plan, None, C.byref(sz)), "stc_plan_save")
    buf = C.create_string_buffer(sz.value)
    check(lib().stc_plan_save(plan, buf, C.byref(sz)), "stc_plan_save")
    return buf.raw[:sz.value]


def stc_plan_load(blob: bytes):
    """Returns (status, plan_handle)."""
    h = C.c_void_p()
    rc = lib().stc_plan_load(blob, len(blob), C.byref(h))
    return rc, h


def stc_plan_upload(plan):
    return lib().stc_plan_upload(plan)


def stc_plan_destroy(plan):
    if plan:
        lib().stc_plan_destroy(plan)


def stc_factor_bytes(plan, batch):
    return int(lib().stc_factor_bytes(plan, int(batch)))


def stc_workspace_bytes(plan, batch):
    return int(lib().stc_workspace_bytes(plan, int(batch)))


def stc_factorize(plan, d_values, batch, d_factor, d_work, d_info, stream=None):
    return lib().stc_factorize(plan, _in_ptr(d_values), int(batch), _dev_ptr(d_factor), _dev_ptr(d_work),
                               _dev_ptr(d_info), _stream(stream))


def stc_scatter_values(plan, d_values, batch, d_factor, stream=None):
    return lib().stc_scatter_values(plan, _in_ptr(d_values), int(batch), _dev_ptr(d_factor), _stream(stream))


def stc_factorize_scattered(plan, batch, d_factor, d_work, d_info, stream=None):
    return lib().stc_factorize_scattered(plan, int(batch), _dev_ptr(d_factor), _dev_ptr(d_work),
                                         _dev_ptr(d_info), _stream(stream))


def stc_sync_status(d_work, stream=None):
    return lib().stc_sync_status(_dev_ptr(d_work), _stream(stream))


def stc_plan_sync_status(plan, stream=None):
    return lib().stc_plan_sync_status(plan, _stream(stream))


def stc_logdet(plan, d_factor, batch, d_logdet, stream=None):
    return lib().stc_logdet(plan, _dev_ptr(d_factor), int(batch), _dev_ptr(d_logdet), _stream(stream))


def stc_solve(plan, d_factor, batch, nrhs, d_b, d_x, d_work, stream=None):
    return lib().stc_solve(plan, _dev_ptr(d_factor), int(batch), int(nrhs), _dev_ptr(d_b), _dev_ptr(d_x),
                           _dev_ptr(d_work), _stream(stream))


def stc_factorize_solve(plan, d_values, batch, nrhs, d_b, d_factor, d_x, d_work, d_info, stream=None):
    return lib().stc_factorize_solve(plan, _in_ptr(d_values), int(batch), int(nrhs), _in_ptr(d_b),
                                     _dev_ptr(d_factor), _dev_ptr(d_x), _dev_ptr(d_work), _dev_ptr(d_info),
                                     _stream(stream))


def stc_factorize_solve_workspace_bytes(plan, batch, nrhs) -> int:
    return int(lib().stc_factorize_solve_workspace_bytes(plan, int(batch), int(nrhs)))


def stc_factorize_forward(plan, d_values, batch, nrhs, d_b, d_factor, d_work, d_info, stream=None):
    return lib().stc_factorize_forward(plan, _in_ptr(d_values), int(batch), int(nrhs), _in_ptr(d_b),
                                       _dev_ptr(d_factor), _dev_ptr(d_work), _dev_ptr(d_info), _stream(stream))


def stc_solve_backward(plan, d_factor, batch, nrhs, d_x, d_work, stream=None):
    return lib().stc_solve_backward(plan, _dev_ptr(d_factor), int(batch), int(nrhs), _dev_ptr(d_x),
                                    _dev_ptr(d_work), _stream(stream))


def stc_factor_to_csc(plan, d_factor, batch, d_Lx, stream=None):
    return lib().stc_factor_to_csc(plan, _dev_ptr(d_factor), int(batch), _dev_ptr(d_Lx), _stream(stream))


def stc_fp64_peak_probe(d_scratch, iters=4096):
    """Returns (status, measured DFMA GFLOP/s)."""
    g = C.c_double(0.0)
    rc = lib().stc_fp64_peak_probe(_dev_ptr(d_scratch), int(d_scratch.numel()), int(iters), C.byref(g))
    return rc, g.value


def stc_factorize_noalloc(plan, d_values, batch, d_factor, d_info, d_status=None, stream=None):
    return lib().stc_factorize_noalloc(plan, _dev_ptr(d_values), int(batch), _dev_ptr(d_factor),
                                       _dev_ptr(d_info), _dev_ptr(d_status), _stream(stream))


def stc_selinv(plan, d_factor, batch, d_sigma, d_work, stream=None):
    return lib().stc_selinv(plan, _dev_ptr(d_factor), int(batch), _dev_ptr(d_sigma), _dev_ptr(d_work),
                            _stream(stream))


def stc_logdet_backward(plan, d_factor, batch, d_gout, d_gvalues, accumulate, d_sigma, d_work, stream=None):
    return lib().stc_logdet_backward(plan, _dev_ptr(d_factor), int(batch), _dev_ptr(d_gout), _dev_ptr(d_gvalues),
                                     int(accumulate), _dev_ptr(d_sigma), _dev_ptr(d_work), _stream(stream))


def stc_sym_outer_backward(plan, batch, d_u, d_v, d_scale, d_gvalues, accumulate, stream=None):
    return lib().stc_sym_outer_backward(plan, int(batch), _dev_ptr(d_u), _dev_ptr(d_v), _dev_ptr(d_scale),
                                        _dev_ptr(d_gvalues), int(accumulate), _stream(stream))


def stc_quad_form(plan, batch, d_values, d_x, d_out, stream=None):
    return lib().stc_quad_form(plan, int(batch), _dev_ptr(d_values), _dev_ptr(d_x), _dev_ptr(d_out),
                               _stream(stream))


def stc_group_create(plans, batches):
    """Returns (status, group_handle)."""
    n = len(plans)
    arr = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in plans])
    bat = (C.c_int64 * n)(*[int(b) for b in batches])
    h = C.c_void_p()
    rc = lib().stc_group_create(n, arr, bat, C.byref(h))
    return rc, h


def stc_group_workspace_bytes(group):
    return int(lib().stc_group_workspace_bytes(group))


def stc_factorize_group(group, d_values, d_factor, d_info, d_work, stream=None):
    n = len(d_values)
    pv = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_values])
    pf = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_factor])
    pi = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_info])
    return lib().stc_factorize_group(group, pv, pf, pi, _dev_ptr(d_work), _stream(stream))


def stc_factorize_mixed(plans, d_values, batches, d_factor, d_info, stream=None):
    n = len(plans)
    pp = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in plans])
    pv = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_values])
    bat = (C.c_int64 * n)(*[int(b) for b in batches])
    pf = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_factor])
    pi = (C.c_void_p * n)(*[_dev_ptr(t).value for t in d_info])
    return lib().stc_factorize_mixed(n, pp, pv, bat, pf, pi, _stream(stream))


def stc_quad_backward(plan, batch, d_x, d_gout, d_gvalues, accumulate, stream=None):
    return lib().stc_quad_backward(plan, int(batch), _dev_ptr(d_x), _dev_ptr(d_gout), _dev_ptr(d_gvalues),
                                   int(accumulate), _stream(stream))


def stc_group_destroy(group):
    if group:
        lib().stc_group_destroy(group)
