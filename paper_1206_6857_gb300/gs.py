"""Thin Python binding of the C ABI in include/gs.h.

Argument marshalling only: every step of the computation runs in the CUDA
library libgs.so.  Device arrays are passed as torch CUDA tensors (their data
pointers and the current torch stream go through the ABI unchanged); host
arrays for gs_sum_host are numpy arrays.  There is no CPU fallback: if the
library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GS_OK = 0
GS_ERR_ARG = -1
GS_ERR_WEIGHT = -2
GS_ERR_NONFINITE = -3
GS_ERR_OOM = -4
GS_ERR_CAPACITY = -5
GS_ERR_TIMEOUT = -6
GS_ERR_CUDA = -7
GS_ERR_UNSUPPORTED = -8

GS_F32 = 0
GS_F64 = 1

GS_SEL_RULE = 0
GS_SEL_MLP = 1
GS_SEL_FD_ONLY = 2
GS_SEL_EXHAUSTIVE = 3

GS_COST_DEFAULT = (32.0, 32.0, 32.0, 1.0)     # c_DH, c_DL, c_H2L, c_Direct weights
GS_FLAG_NO_MERGE = 1


class gs_opts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("plimit", ctypes.c_int32),
                ("selector", ctypes.c_int32), ("no_tokens", ctypes.c_int32),
                ("floor_log2", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("pair_capacity", ctypes.c_int64), ("cost_weight", ctypes.c_double * 4),
                ("reserved", ctypes.c_int64 * 4)]


GS_PH_INGEST, GS_PH_TREE, GS_PH_FRONTIER, GS_PH_SERIES, GS_PH_BASE, GS_PH_DOWN, GS_PH_OTHER = range(7)
GS_NPHASE = 8
PHASE_NAMES = ["ingest", "tree", "frontier", "series", "base", "down", "other", "spare"]


class gs_stats(ctypes.Structure):
    _fields_ = [("pairs_fd", ctypes.c_int64), ("pairs_dh", ctypes.c_int64),
                ("pairs_dl", ctypes.c_int64), ("pairs_h2l", ctypes.c_int64),
                ("pairs_base", ctypes.c_int64), ("pairs_split", ctypes.c_int64),
                ("point_pairs_base", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("launches_base", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("retries", ctypes.c_int32), ("fp32_rel_bound", ctypes.c_double),
                ("eps_traversal", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_phase", ctypes.c_double * GS_NPHASE), ("reserved", ctypes.c_double * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "ms_phase")}
        d["ms_phase"] = {PHASE_NAMES[i]: self.ms_phase[i] for i in range(GS_NPHASE)}
        return d


class GSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gs error %d: %s" % (code, msg))
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_SUM_ARGS = [_VP, _I64, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int,
             ctypes.c_double, _VP, _VP, _VP, _VP]

# every symbol include/gs.h declares, with its ctypes signature
SIGNATURES = {
    "gs_version": (ctypes.c_char_p, []),
    "gs_last_error": (ctypes.c_char_p, []),
    "gs_opts_default": (ctypes.c_int, [_VP]),
    "gs_sum": (ctypes.c_int, _SUM_ARGS),
    "gs_sum_host": (ctypes.c_int, _SUM_ARGS),
    "gs_probe_rates": (ctypes.c_int, [_VP, _VP, _VP]),
    "gs_sum_trace": (ctypes.c_int, _SUM_ARGS + [_VP, _I64, _VP, _VP, _VP]),
    "gs_sum_exhaustive_noalloc": (ctypes.c_int, [_VP, _I64, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, _VP,
                                                  ctypes.c_int, _VP, _VP]),
    "gs_lscv": (ctypes.c_int, [_VP, _I64, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_double,
                               _VP, _VP, _VP, _VP, _VP]),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libgs.so (raises if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libgs.so is not built; run paper_1206_6857_gb300.build.build() "
                               "(or __graft_entry__.build()) first")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def gs_version() -> str:
    return load().gs_version().decode()


def gs_last_error() -> str:
    return load().gs_last_error().decode()


def gs_opts_default() -> gs_opts:
    o = gs_opts()
    _check(load().gs_opts_default(ctypes.byref(o)))
    return o


def _check(rc):
    if rc != GS_OK:
        raise GSError(rc, gs_last_error())
    return rc


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return GS_F32
    if t.dtype == torch.float64:
        return GS_F64
    raise TypeError("points must be float32 or float64, got %s" % t.dtype)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def gs_sum(queries, refs, weights, h, eps, out=None, opts: gs_opts | None = None, stream=None,
           stats: gs_stats | None = None, raise_on_error: bool = True):
    """G~(x_q; h_j) for torch CUDA tensors queries (M x D), refs (N x D),
    weights (N, float32); h is a host sequence of bandwidths.  Pass the same
    tensor as queries and refs for the monochromatic problem.  Returns out
    (M x nh float64 CUDA tensor)."""
    import torch
    assert queries.is_cuda and refs.is_cuda and weights.is_cuda
    assert queries.is_contiguous() and refs.is_contiguous() and weights.is_contiguous()
    assert weights.dtype == torch.float32
    M, D = queries.shape
    N = refs.shape[0]
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    if out is None:
        out = torch.empty((M, hh.size), dtype=torch.float64, device=queries.device)
    rc = load().gs_sum(_VP(queries.data_ptr()), M, _VP(refs.data_ptr()), _VP(weights.data_ptr()), N, D,
                       _dtype_code(queries), hh.ctypes.data, hh.size, float(eps), _VP(out.data_ptr()),
                       ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                       ctypes.byref(stats) if stats is not None else None)
    if raise_on_error:
        _check(rc)
        return out
    return rc, out


def gs_sum_trace(queries, refs, weights, h, eps, opts: gs_opts | None = None, stream=None,
                 trace_cap: int = 1 << 22, stats: gs_stats | None = None):
    """gs_sum (eps > 0) plus the traversal record: returns (out, trace, qperm,
    rperm) with trace an (n, 4) int32 CUDA tensor of (query node, reference
    node, bandwidth, action | order << 8 | iteration << 16)."""
    import torch
    M, D = queries.shape
    N = refs.shape[0]
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    dev = queries.device
    out = torch.empty((M, hh.size), dtype=torch.float64, device=dev)
    tr = torch.empty((trace_cap, 4), dtype=torch.int32, device=dev)
    qperm = torch.empty(M, dtype=torch.int32, device=dev)
    rperm = torch.empty(N, dtype=torch.int32, device=dev)
    n = ctypes.c_int64()
    _check(load().gs_sum_trace(_VP(queries.data_ptr()), M, _VP(refs.data_ptr()), _VP(weights.data_ptr()), N, D,
                               _dtype_code(queries), hh.ctypes.data, hh.size, float(eps), _VP(out.data_ptr()),
                               ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                               ctypes.byref(stats) if stats is not None else None, _VP(tr.data_ptr()), trace_cap,
                               ctypes.byref(n), _VP(qperm.data_ptr()), _VP(rperm.data_ptr())))
    if n.value > trace_cap:
        raise GSError(GS_ERR_CAPACITY, "trace of %d records exceeds trace_cap=%d" % (n.value, trace_cap))
    return out, tr[:n.value], qperm, rperm


def gs_sum_exhaustive_noalloc(queries, refs, weights, h, out=None, stream=None, raise_on_error: bool = True):
    """Exhaustive sums through the allocation-free entry point (its scratch is a
    fixed array inside the library); same tensors as gs_sum with eps = 0."""
    import torch
    assert queries.is_cuda and refs.is_cuda and weights.is_cuda
    M, D = queries.shape
    N = refs.shape[0]
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    if out is None:
        out = torch.empty((M, hh.size), dtype=torch.float64, device=queries.device)
    rc = load().gs_sum_exhaustive_noalloc(_VP(queries.data_ptr()), M, _VP(refs.data_ptr()),
                                          _VP(weights.data_ptr()), N, D, _dtype_code(queries), hh.ctypes.data,
                                          hh.size, _VP(out.data_ptr()), _stream_ptr(stream))
    if raise_on_error:
        _check(rc)
        return out
    return rc, out


def gs_lscv(points, weights, h, eps, opts: gs_opts | None = None, stream=None, stats: gs_stats | None = None):
    """LSCV scores (and their eps-implied error bounds) for every bandwidth in
    h, from a torch CUDA tensor of points (N x D) and float32 weights."""
    assert points.is_cuda and weights.is_cuda and points.is_contiguous() and weights.is_contiguous()
    N, D = points.shape
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    score = np.empty(hh.size)
    err = np.empty(hh.size)
    _check(load().gs_lscv(_VP(points.data_ptr()), N, D, _dtype_code(points), _VP(weights.data_ptr()),
                          hh.ctypes.data, hh.size, float(eps), score.ctypes.data, err.ctypes.data,
                          ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                          ctypes.byref(stats) if stats is not None else None))
    return score, err


def gs_sum_host(queries: np.ndarray, refs: np.ndarray, weights: np.ndarray, h, eps,
                out: np.ndarray | None = None, opts: gs_opts | None = None, stream=None,
                stats: gs_stats | None = None):
    """gs_sum on host (numpy) arrays; the library copies in and out."""
    mono = queries is refs
    q = np.ascontiguousarray(queries)
    r = q if mono else np.ascontiguousarray(refs)
    assert q.dtype == r.dtype and q.dtype in (np.float32, np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    M, D = q.shape
    N = r.shape[0]
    if out is None:
        out = np.empty((M, hh.size), dtype=np.float64)
    sp = None if stream is None else _stream_ptr(stream)
    _check(load().gs_sum_host(q.ctypes.data, M, r.ctypes.data, w.ctypes.data, N, D,
                              GS_F64 if q.dtype == np.float64 else GS_F32, hh.ctypes.data, hh.size,
                              float(eps), out.ctypes.data,
                              ctypes.byref(opts) if opts is not None else None, sp,
                              ctypes.byref(stats) if stats is not None else None))
    return out


def gs_probe_rates(stream=None):
    """(ex2 lanes, FFMA lanes) per SM per SM clock, measured on this device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().gs_probe_rates(ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)))
    return a.value, b.value
