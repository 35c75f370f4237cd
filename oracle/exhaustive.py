"""FP64 exhaustive Gaussian sum (the definition of Section 1), via the C
oracle in exhaustive.c.  TEST INFRASTRUCTURE ONLY.

gauss_sum(queries, refs, w, h, skip_self=False) -> (M, nh) float64 array with
G(x_q; h_j) = sum_r w_r exp(-||x_q - x_r||^2 / (2 h_j^2)).
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        lib.oracle_gauss_sum.restype = ctypes.c_int
        lib.oracle_gauss_sum.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def gauss_sum(queries, refs, w, h, skip_self: bool = False) -> np.ndarray:
    q = np.ascontiguousarray(queries, dtype=np.float64)
    r = np.ascontiguousarray(refs, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    h = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    if q.ndim == 1:
        q = q[:, None]
    if r.ndim == 1:
        r = r[:, None]
    M, D = q.shape
    N = r.shape[0]
    assert r.shape[1] == D and w.shape == (N,)
    if skip_self:
        assert M == N, "skip_self needs queries == refs"
    out = np.empty((M, h.size), dtype=np.float64)
    rc = _load().oracle_gauss_sum(q.ctypes.data, M, r.ctypes.data, w.ctypes.data, N, D,
                                  h.ctypes.data, h.size, int(skip_self), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_gauss_sum: unsupported number of bandwidths %d" % h.size)
    return out
