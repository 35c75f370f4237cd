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
