"""Expanded-distance base case (FP32 points, D <= 8).

Leaf pairs whose reference leaf passes the error guard at a bandwidth take
||q - r||^2 = (|v|^2 - 2 u.v) + |u|^2 about the reference leaf's centre; the
rest stay with the direct kernel.  Against the FP64 oracle:
* every result within eps, with the path on and off (GS_FLAG_NO_XP), and the
  path actually summing terms;
* a traversal that prunes nothing (every leaf pair summed in the base case):
  the whole sum within the FP32 charge the call reports, which includes the
  path's share (the bit-exact traversal cases with leaves of 64 and 128
  points check that share against the CPU traversal).
"""
import numpy as np
import pytest

from helpers import rel_err
from oracle import dualtree as T
from oracle import exhaustive as oracle_ex
from workloads import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    from paper_1206_6857_gb300 import build, gs as _gs
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    _gs.load()
    return _gs


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _opts(gs, leaf, flags=0, selector=None):
    o = gs.gs_opts_default()
    o.leaf_size = leaf
    o.flags = flags
    if selector is not None:
        o.selector = selector
    return o


@pytest.mark.parametrize("cfg,leaf", [(2, 64), (3, 128)])
def test_expanded_path_within_eps(gs, cfg, leaf):
    wl = synth.config2(0.02) if cfg == 2 else synth.config3(0.02, eps=1e-3)
    tq, tw = _dev(wl.queries), _dev(wl.weights)
    st = gs.gs_stats()
    got = gs.gs_sum(tq, tq, tw, wl.h, wl.eps, opts=_opts(gs, leaf), stats=st).cpu().numpy()
    assert st.point_pairs_xp > 0, st.as_dict()
    st2 = gs.gs_stats()
    off = gs.gs_sum(tq, tq, tw, wl.h, wl.eps, opts=_opts(gs, leaf, gs.GS_FLAG_NO_XP), stats=st2).cpu().numpy()
    assert st2.point_pairs_xp == 0
    assert st.fp32_rel_bound - st2.fp32_rel_bound == pytest.approx(T.xp_rho(), rel=1e-9)
    exact = oracle_ex.gauss_sum(wl.queries, wl.refs, wl.weights, wl.h)
    W = float(wl.weights.astype(np.float64).sum())
    assert rel_err(got, exact, W).max() <= wl.eps
    assert rel_err(off, exact, W).max() <= wl.eps


@pytest.mark.parametrize("D,offset", [(2, 0.0), (3, 0.0), (5, 1000.0), (8, 0.0)])
def test_expanded_terms_match_the_exhaustive_sum(gs, D, offset):
    """Nothing pruned (exhaustive selector, large bandwidths): the base case
    carries the whole sum, mostly on the expanded path; uneven weights (l != 0)
    and, for one case, coordinates offset far from the origin."""
    q, r, w = synth.small_random(40 + D, 6000, D)
    q = (q + np.float32(offset)).astype(np.float32)
    diam = synth.bbox_diagonal(q)
    h = np.array([0.05, 0.1, 0.3, 0.8]) * diam
    st = gs.gs_stats()
    got = gs.gs_sum(_dev(q), _dev(q), _dev(w), h, 1e-3, opts=_opts(gs, 64, selector=gs.GS_SEL_EXHAUSTIVE),
                    stats=st).cpu().numpy()
    assert st.point_pairs_xp > 0.5 * st.point_pairs_base, st.as_dict()
    exact = oracle_ex.gauss_sum(q, q, w, h)
    err = np.abs(got - exact) / exact
    assert err.max() <= st.fp32_rel_bound, (err.max(), st.fp32_rel_bound)
