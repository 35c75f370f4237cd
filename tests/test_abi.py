"""The C-ABI library loads and exports every entry point include/gs.h
declares; argument checks that need no GPU return the documented codes."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1206_6857_gb300 import build, gs
    build.build()
    return gs.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1206_6857_gb300 import gs
    names = _declared_functions()
    assert "gs_sum" in names and "gs_version" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gs.SIGNATURES), "binding and header disagree"


def test_version_and_defaults(lib):
    from paper_1206_6857_gb300 import gs
    assert "sm_103a" in gs.gs_version()
    o = gs.gs_opts_default()
    assert o.leaf_size == 32 and o.floor_log2 == -40 and o.selector == gs.GS_SEL_RULE


def test_argument_errors_need_no_gpu(lib):
    from paper_1206_6857_gb300 import gs
    h = np.array([0.1])
    buf = ctypes.c_void_p(16)        # never dereferenced: argument checks run first
    call = lambda **kw: lib.gs_sum(kw.get("q", buf), kw.get("M", 10), kw.get("r", buf),
                                   kw.get("w", buf), kw.get("N", 10), kw.get("D", 3),
                                   kw.get("dtype", gs.GS_F32), kw.get("h", h.ctypes.data),
                                   kw.get("nh", 1), kw.get("eps", 0.01), kw.get("out", buf),
                                   None, None, None)
    assert call(q=None) == gs.GS_ERR_ARG
    assert call(M=0) == gs.GS_ERR_ARG
    assert call(D=0) == gs.GS_ERR_ARG and call(D=33) == gs.GS_ERR_ARG
    assert call(dtype=7) == gs.GS_ERR_ARG
    assert call(nh=0) == gs.GS_ERR_ARG and call(nh=65) == gs.GS_ERR_ARG
    assert call(eps=1.0) == gs.GS_ERR_ARG and call(eps=-0.1) == gs.GS_ERR_ARG
    bad_h = np.array([-1.0])
    assert call(h=bad_h.ctypes.data) == gs.GS_ERR_ARG
    inf_h = np.array([np.inf])
    assert call(h=inf_h.ctypes.data) == gs.GS_ERR_ARG
    assert "outside" in gs.gs_last_error() or "bandwidth" in gs.gs_last_error()


def _cpu_args(M=5, N=7, D=3, dt=None):
    import torch
    dt = dt or torch.float32
    return torch.zeros(M, D, dtype=dt), torch.zeros(N, D, dtype=dt), torch.ones(N, dtype=torch.float32)


MISMATCHES = [
    ("refs dtype", lambda q, r, w, t: (q, r.to(t.float64), w, None), "refs dtype"),
    ("refs width", lambda q, r, w, t: (q, t.zeros(r.shape[0], 4), w, None), "columns"),
    ("weights dtype", lambda q, r, w, t: (q, r, w.to(t.float64), None), "weights must be float32"),
    ("weights length", lambda q, r, w, t: (q, r, w[:-1], None), "weights must have shape"),
    ("weights 2-D", lambda q, r, w, t: (q, r, w[:, None], None), "weights must have shape"),
    ("points dtype", lambda q, r, w, t: (q.to(t.float16), r.to(t.float16), w, None), "float32 or float64"),
    ("points 1-D", lambda q, r, w, t: (q.reshape(-1), r, w, None), "2-D"),
    ("non-contiguous", lambda q, r, w, t: (t.zeros(3, 5).t(), r, w, None), "contiguous"),
    ("out dtype", lambda q, r, w, t: (q, r, w, t.zeros(q.shape[0], 2, dtype=t.float32)), "out must be a float64"),
    ("out rows", lambda q, r, w, t: (q, r, w, t.zeros(q.shape[0] - 1, 2, dtype=t.float64)), "shape"),
    ("out columns", lambda q, r, w, t: (q, r, w, t.zeros(q.shape[0], 3, dtype=t.float64)), "shape"),
]


@pytest.mark.parametrize("case", MISMATCHES, ids=lambda c: c[0])
def test_wrappers_refuse_mismatched_arguments(case):
    """A dtype, width, length or output-shape mismatch is refused by the
    binding itself, before a device pointer reaches the library (where it
    would make a kernel read or write past a buffer's end)."""
    import torch
    from paper_1206_6857_gb300 import gs
    _, make, msg = case
    q, r, w, out = make(*_cpu_args(), torch)
    with pytest.raises(ValueError, match=msg):
        gs._check_sum_tensors(q, r, w, 2, out)
    # every public wrapper runs the same check first
    for call in (lambda: gs.gs_sum(q, r, w, [0.1, 0.2], 0.0, out=out),
                 lambda: gs.gs_sum_exhaustive_noalloc(q, r, w, [0.1, 0.2], out=out)):
        with pytest.raises(ValueError, match=msg):
            call()


def test_wrappers_refuse_host_tensors():
    """Matching CPU tensors pass the layout checks and are then refused as
    not being on a CUDA device."""
    from paper_1206_6857_gb300 import gs
    q, r, w = _cpu_args()
    with pytest.raises(ValueError, match="CUDA"):
        gs.gs_sum(q, r, w, [0.1], 1e-2)
    with pytest.raises(ValueError, match="CUDA"):
        gs.gs_sum_exhaustive_noalloc(q, r, w, [0.1])
