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
GS_FLAG_SMALL_EXHAUSTIVE = 2
GS_FLAG_NO_TC = 4
GS_FLAG_BEST_FIRST = 8
GS_SMALL_WORK = 549755813888.0
GS_SMALL_WORK_D2 = 68719476736.0

GS_MLP_NIN = 12
GS_MLP_NOUT = 5
GS_MLP_NPARAM = 5341


class gs_opts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("plimit", ctypes.c_int32),
                ("selector", ctypes.c_int32), ("no_tokens", ctypes.c_int32),
                ("floor_log2", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("pair_capacity", ctypes.c_int64), ("cost_weight", ctypes.c_double * 4),
                ("selector_params", ctypes.c_void_p), ("small_work", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 2)]


GS_PH_INGEST, GS_PH_TREE, GS_PH_FRONTIER, GS_PH_SERIES, GS_PH_BASE, GS_PH_DOWN, GS_PH_OTHER, GS_PH_BASE_TC = range(8)
GS_NPHASE = 8
PHASE_NAMES = ["ingest", "tree", "frontier", "series", "base", "down", "other", "base_tc"]


class gs_problem(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_void_p), ("M", ctypes.c_int64), ("refs", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("N", ctypes.c_int64), ("D", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("h", ctypes.c_void_p), ("nh", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("eps", ctypes.c_double), ("out", ctypes.c_void_p)]


class gs_stats(ctypes.Structure):
    _fields_ = [("pairs_fd", ctypes.c_int64), ("pairs_dh", ctypes.c_int64),
                ("pairs_dl", ctypes.c_int64), ("pairs_h2l", ctypes.c_int64),
                ("pairs_base", ctypes.c_int64), ("pairs_split", ctypes.c_int64),
                ("point_pairs_base", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("launches_base", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("retries", ctypes.c_int32), ("fp32_rel_bound", ctypes.c_double),
                ("eps_traversal", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_phase", ctypes.c_double * GS_NPHASE), ("ms_series", ctypes.c_double * 3),
                ("point_pairs_tc", ctypes.c_int64), ("ms_base_kernels", ctypes.c_double * 2)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("reserved", "ms_phase", "ms_series", "ms_base_kernels")}
        d["ms_base_kernels"] = [self.ms_base_kernels[0], self.ms_base_kernels[1]]
        d["ms_phase"] = {PHASE_NAMES[i]: self.ms_phase[i] for i in range(GS_NPHASE)}
        d["ms_series"] = {"dh": self.ms_series[0], "dl": self.ms_series[1], "h2l": self.ms_series[2]}
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
    "gs_trim_memory": (ctypes.c_int, [ctypes.c_size_t]),
    "gs_tc_dot_check": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    "gs_pool_bytes": (ctypes.c_int, [_VP, _VP]),
    "gs_sum_trace": (ctypes.c_int, _SUM_ARGS + [_VP, _I64, _VP, _VP, _VP]),
    "gs_sum_exhaustive_noalloc": (ctypes.c_int, [_VP, _I64, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, _VP,
                                                  ctypes.c_int, _VP, _VP]),
    "gs_lscv": (ctypes.c_int, [_VP, _I64, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_double,
                               _VP, _VP, _VP, _VP, _VP]),
    "gs_lscv_host": (ctypes.c_int, [_VP, _I64, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int,
                                    ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
    "gs_mlp_forward": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP]),
    "gs_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "gs_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_int, _VP, _VP]),
    "gs_sum_batched": (ctypes.c_int, [ctypes.c_int, _VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "gs_debug_fail_alloc": (None, [ctypes.c_longlong]),
    "gs_build_tree": (ctypes.c_int, [_VP, ctypes.c_int, _I64, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "gs_tree_free": (None, [_VP]),
    "gs_sum_trees": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP, _VP, _VP, _VP]),
    "gs_lscv_trees": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
    "gs_selector_samples": (ctypes.c_int, [_VP, _I64, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, _VP,
                                           ctypes.c_int, ctypes.c_double, _VP, _VP, _VP, _VP, _VP, _I64, _VP,
                                           _VP, _VP]),
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


def _check_sum_tensors(queries, refs, weights, nh, out=None):
    """Refuse arguments whose sizes or element types disagree before any
    pointer reaches the library (a mismatch there would make a kernel read
    or write past the end of a buffer): 2-D contiguous point tensors of one
    floating type and width D, weights (N,) float32, out (M, nh) float64 on
    the same device.  The device check comes last, so the layout checks run
    on CPU tensors too.  Raises ValueError."""
    import torch
    for name, t in (("queries", queries), ("refs", refs), ("weights", weights)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
    if queries.dim() != 2 or refs.dim() != 2:
        raise ValueError("queries and refs must be 2-D (points x D)")
    if queries.dtype not in (torch.float32, torch.float64):
        raise ValueError("points must be float32 or float64, got %s" % queries.dtype)
    if refs.dtype != queries.dtype:
        raise ValueError("refs dtype %s differs from queries dtype %s" % (refs.dtype, queries.dtype))
    if refs.shape[1] != queries.shape[1]:
        raise ValueError("refs have D=%d columns, queries D=%d" % (refs.shape[1], queries.shape[1]))
    if weights.dtype != torch.float32:
        raise ValueError("weights must be float32, got %s" % weights.dtype)
    if weights.dim() != 1 or weights.shape[0] != refs.shape[0]:
        raise ValueError("weights must have shape (%d,), got %s" % (refs.shape[0], tuple(weights.shape)))
    if not (queries.is_contiguous() and refs.is_contiguous() and weights.is_contiguous()):
        raise ValueError("queries, refs and weights must be contiguous")
    if out is not None:
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float64:
            raise ValueError("out must be a float64 tensor")
        if tuple(out.shape) != (queries.shape[0], nh) or not out.is_contiguous():
            raise ValueError("out must be contiguous with shape (%d, %d), got %s"
                             % (queries.shape[0], nh, tuple(out.shape)))
    devs = {queries.device, refs.device, weights.device} | ({out.device} if out is not None else set())
    if len(devs) != 1 or not queries.is_cuda:
        raise ValueError("queries, refs, weights and out must be CUDA tensors on one device")


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
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    _check_sum_tensors(queries, refs, weights, hh.size, out)
    M, D = queries.shape
    N = refs.shape[0]
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
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    _check_sum_tensors(queries, refs, weights, hh.size)
    M, D = queries.shape
    N = refs.shape[0]
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
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    _check_sum_tensors(queries, refs, weights, hh.size, out)
    M, D = queries.shape
    N = refs.shape[0]
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
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    _check_sum_tensors(points, points, weights, hh.size)
    N, D = points.shape
    score = np.empty(hh.size)
    err = np.empty(hh.size)
    _check(load().gs_lscv(_VP(points.data_ptr()), N, D, _dtype_code(points), _VP(weights.data_ptr()),
                          hh.ctypes.data, hh.size, float(eps), score.ctypes.data, err.ctypes.data,
                          ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                          ctypes.byref(stats) if stats is not None else None))
    return score, err


def gs_lscv_host(points: np.ndarray, weights: np.ndarray, h, eps, opts: gs_opts | None = None, stream=None,
                 stats: gs_stats | None = None):
    """gs_lscv on host (numpy) arrays; the library copies the inputs in.
    Returns (score, err) host arrays."""
    p = np.ascontiguousarray(points)
    if p.ndim != 2 or p.dtype not in (np.float32, np.float64):
        raise ValueError("points must be a 2-D float32 or float64 array")
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if w.shape != (p.shape[0],):
        raise ValueError("weights must have shape (%d,)" % p.shape[0])
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    score = np.empty(hh.size)
    err = np.empty(hh.size)
    sp = None if stream is None else _stream_ptr(stream)
    _check(load().gs_lscv_host(p.ctypes.data, p.shape[0], p.shape[1], GS_F64 if p.dtype == np.float64 else GS_F32,
                               w.ctypes.data, hh.ctypes.data, hh.size, float(eps), score.ctypes.data,
                               err.ctypes.data, ctypes.byref(opts) if opts is not None else None, sp,
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


def gs_tc_dot_check(U: np.ndarray, V: np.ndarray, stream=None):
    """Raw tensor-core accumulators (3 x 128 x N float32) of the base case's
    fixed-point cross term for integer matrices U (128 x 16) and V (N x 16)."""
    U = np.ascontiguousarray(U, dtype=np.int32)
    V = np.ascontiguousarray(V, dtype=np.int32)
    if U.shape != (128, 16) or V.ndim != 2 or V.shape[1] != 16:
        raise ValueError("U must be 128 x 16 and V N x 16")
    N = V.shape[0]
    P = np.empty((3, 128, N), dtype=np.float32)
    _check(load().gs_tc_dot_check(U.ctypes.data, V.ctypes.data, N, P.ctypes.data, _stream_ptr(stream)))
    return P


def gs_trim_memory(keep_bytes=0):
    """Return all but keep_bytes of the library's device pool to the CUDA driver."""
    _check(load().gs_trim_memory(int(keep_bytes)))


def gs_pool_bytes():
    """(reserved, used) bytes of the library's device pool."""
    r, u = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().gs_pool_bytes(ctypes.byref(r), ctypes.byref(u)))
    return r.value, u.value


# ---------------------------------------------------------------------------
# learned pair selector
# ---------------------------------------------------------------------------
def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def gs_mlp_forward(params, x, stream=None):
    """Selector scores (n x 5 float32 CUDA tensor) of x (n x 12 float32)."""
    import torch
    assert params.is_cuda and params.dtype == torch.float32 and params.numel() == GS_MLP_NPARAM
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.shape[1] == GS_MLP_NIN
    out = torch.empty((x.shape[0], GS_MLP_NOUT), dtype=torch.float32, device=x.device)
    _check(load().gs_mlp_forward(_ptr(params), _ptr(x), x.shape[0], _ptr(out), _stream_ptr(stream)))
    return out


def gs_mlp_loss_grad(params, x, y, s=None, stream=None):
    """(loss, grad): mean weighted softmax cross entropy and its FP64 gradient (CUDA tensors)."""
    import torch
    grad = torch.empty(GS_MLP_NPARAM, dtype=torch.float64, device=x.device)
    loss = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(load().gs_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(y), _ptr(s), x.shape[0], _ptr(grad), _ptr(loss),
                                   _stream_ptr(stream)))
    return loss, grad


def gs_mlp_train(params, x, y, s=None, epochs=10, batch=4096, lr=1e-3, seed=0, set_norm=True, stream=None):
    """Adam training of params (updated in place); returns the per-epoch mean losses."""
    losses = (ctypes.c_double * max(epochs, 1))()
    _check(load().gs_mlp_train(_ptr(params), _ptr(x), _ptr(y), _ptr(s), x.shape[0], int(epochs), int(batch),
                               float(lr), ctypes.c_uint64(seed), int(bool(set_norm)), losses, _stream_ptr(stream)))
    return [losses[i] for i in range(epochs)]


def gs_selector_samples(queries, refs, weights, h, eps, unit_cost, cap, opts: gs_opts | None = None, stream=None):
    """Selector training samples of one problem: (x, y, s, model_cost) CUDA tensors
    truncated to the sample count; model_cost = (cheapest policy, FD-only policy)."""
    import torch
    h = np.ascontiguousarray(h, dtype=np.float64)
    M, D = queries.shape
    N = refs.shape[0]
    dev = queries.device
    x = torch.empty((max(cap, 1), GS_MLP_NIN), dtype=torch.float32, device=dev)
    y = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    s = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    assert len(unit_cost) == 6
    uc = (ctypes.c_double * 6)(*[float(v) for v in unit_cost])
    n = ctypes.c_int64(0)
    mc = (ctypes.c_double * 2)()
    _check(load().gs_selector_samples(_ptr(queries), M, _ptr(refs), _ptr(weights), N, D, _dtype_code(queries),
                                      h.ctypes.data_as(_VP), len(h), float(eps),
                                      ctypes.byref(opts) if opts is not None else None, uc, _ptr(x), _ptr(y),
                                      _ptr(s), cap, ctypes.byref(n), mc, _stream_ptr(stream)))
    k = n.value
    return x[:k], y[:k], s[:k], (mc[0], mc[1])


def gs_sum_batched(problems, opts: gs_opts | None = None, nworkers: int = 0, stream=None,
                   stats: gs_stats | None = None, raise_on_error: bool = True):
    """problems: sequence of (queries, refs, weights, h, eps) with torch CUDA
    tensors (queries may be refs).  Returns the list of outputs (M x nh
    float64 CUDA tensors) and the per-problem status codes."""
    import torch
    n = len(problems)
    arr = (gs_problem * max(n, 1))()
    outs, keep = [], []
    for i, (q, r, w, h, eps) in enumerate(problems):
        hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
        _check_sum_tensors(q, r, w, hh.size)
        keep.append(hh)
        out = torch.empty((q.shape[0], hh.size), dtype=torch.float64, device=q.device)
        outs.append(out)
        arr[i] = gs_problem(q.data_ptr(), q.shape[0], r.data_ptr(), w.data_ptr(), r.shape[0], q.shape[1],
                            _dtype_code(q), hh.ctypes.data, hh.size, 0, float(eps), out.data_ptr())
    status = (ctypes.c_int32 * max(n, 1))()
    rc = load().gs_sum_batched(n, arr, ctypes.byref(opts) if opts is not None else None, int(nworkers),
                               _stream_ptr(stream), ctypes.byref(stats) if stats is not None else None, status)
    if raise_on_error:
        _check(rc)
    return outs, [status[i] for i in range(n)]


class Tree:
    """A built kd-tree (gs_build_tree); freed with close() or when collected."""

    def __init__(self, points, weights=None, opts: gs_opts | None = None, stream=None):
        if weights is not None:
            _check_sum_tensors(points, points, weights, 1)
        else:
            import torch
            ok = (isinstance(points, torch.Tensor) and points.dim() == 2 and points.is_contiguous()
                  and points.dtype in (torch.float32, torch.float64) and points.is_cuda)
            if not ok:
                raise ValueError("points must be a contiguous 2-D float32/float64 CUDA tensor")
        self.M = points.shape[0]
        self.D = points.shape[1]
        self.device = points.device
        self._h = ctypes.c_void_p()
        _check(load().gs_build_tree(_ptr(points), _dtype_code(points), points.shape[0], points.shape[1],
                                    _ptr(weights), ctypes.byref(opts) if opts is not None else None,
                                    _stream_ptr(stream), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            load().gs_tree_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_lscv_trees(tree: Tree, h, eps, opts: gs_opts | None = None, stream=None, stats: gs_stats | None = None):
    """LSCV scores and their eps-implied bounds for the bandwidths h (at most
    32) on a built reference tree; returns (score, err) host arrays."""
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    score = np.empty(hh.size)
    err = np.empty(hh.size)
    _check(load().gs_lscv_trees(tree._h, hh.ctypes.data, hh.size, float(eps), score.ctypes.data, err.ctypes.data,
                                ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                                ctypes.byref(stats) if stats is not None else None))
    return score, err


def gs_sum_trees(qtree: Tree, rtree: Tree, h, eps, out=None, opts: gs_opts | None = None, stream=None,
                 stats: gs_stats | None = None):
    """gs_sum on built trees (qtree is rtree: monochromatic); returns out (M x nh float64)."""
    import torch
    hh = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    if out is None:
        out = torch.empty((qtree.M, hh.size), dtype=torch.float64, device=qtree.device)
    _check(load().gs_sum_trees(qtree._h, rtree._h, hh.ctypes.data, hh.size, float(eps), _ptr(out),
                               ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream),
                               ctypes.byref(stats) if stats is not None else None))
    return out
