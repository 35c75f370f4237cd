"""Tensor-core base case (9 <= D <= 16).

* The fixed-point cross term: three base-2^10 digits per coordinate, products
  accumulated in FP32 on the tensor cores.  Every accumulator is an integer
  below 2^24, so gs_tc_dot_check's raw accumulators must equal the integer
  sums exactly, extremes of the digit range included.
* The base case with the cross term on the tensor cores against the direct
  FP32 kernel (GS_FLAG_NO_TC) and against the FP64 oracle: every result
  within eps, and the tensor-core path actually summed terms.
"""
import numpy as np
import pytest

from helpers import rel_err
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


def _digits(X):
    """Balanced base-2^10 digits (U2, U1, U0) of int64 values, written from
    the definition U = U2 2^20 + U1 2^10 + U0, U0 and U1 in [-512, 511]."""
    X = X.astype(np.int64)
    d0 = np.mod(X + 512, 1024) - 512
    t = (X - d0) // 1024
    d1 = np.mod(t + 512, 1024) - 512
    d2 = (t - d1) // 1024
    assert np.all(d2 * 2 ** 20 + d1 * 2 ** 10 + d0 == X)
    return d2, d1, d0


@pytest.mark.parametrize("N", [16, 32, 128])
def test_fixed_point_cross_term_is_exact(gs, N):
    rng = np.random.default_rng(N)
    lim = 2 ** 29
    U = rng.integers(-lim, lim + 1, (128, 16))
    V = rng.integers(-lim, lim + 1, (N, 16))
    # extremes: the largest magnitudes and the digit-range edges
    U[0, :] = lim
    U[1, :] = -lim
    U[2, :] = 2 ** 20 - 1
    V[0, :] = lim
    V[1, :] = -(2 ** 19) - 512
    V[2, ::2] = -lim
    P = gs.gs_tc_dot_check(U, V)
    u2, u1, u0 = _digits(U)
    v2, v1, v0 = _digits(V)
    want = [u2 @ v2.T, u2 @ v1.T + u1 @ v2.T, u2 @ v0.T + u1 @ v1.T + u0 @ v2.T]
    for g in range(3):
        assert np.abs(want[g]).max() < 2 ** 24
        assert np.array_equal(P[g].astype(np.int64), want[g]), g


@pytest.mark.parametrize("D,scale", [(16, 0.005), (12, 0.004), (9, 0.004)])
def test_tensor_core_base_case_within_eps(gs, D, scale):
    """C4-shaped bichromatic data (projected to D dimensions for D < 16): the
    tensor-core path against the direct kernel and the FP64 oracle."""
    wl = synth.config4(scale)
    q = np.ascontiguousarray(wl.queries[:, :D])
    r = np.ascontiguousarray(wl.refs[:, :D])
    h = synth.log_bandwidths(synth.bbox_diagonal(r), 8, 1e-2, 1.0)
    tq, tr, tw = _dev(q), _dev(r), _dev(wl.weights)
    o = gs.gs_opts_default()
    o.leaf_size = 64
    st = gs.gs_stats()
    got = gs.gs_sum(tq, tr, tw, h, wl.eps, opts=o, stats=st).cpu().numpy()
    assert st.point_pairs_tc > 0, st.as_dict()
    o2 = gs.gs_opts_default()
    o2.leaf_size = 64
    o2.flags = gs.GS_FLAG_NO_TC
    st2 = gs.gs_stats()
    direct = gs.gs_sum(tq, tr, tw, h, wl.eps, opts=o2, stats=st2).cpu().numpy()
    assert st2.point_pairs_tc == 0
    assert st.fp32_rel_bound > st2.fp32_rel_bound        # the tensor-core charge
    exact = oracle_ex.gauss_sum(q, r, wl.weights, h)
    W = float(wl.weights.astype(np.float64).sum())
    assert rel_err(got, exact, W).max() <= wl.eps
    assert rel_err(direct, exact, W).max() <= wl.eps


def test_tensor_core_terms_match_the_exhaustive_sum(gs):
    """A traversal with almost nothing pruned (eps tiny, large bandwidths):
    the base case carries nearly all of the sum, so its tensor-core arithmetic
    is compared with the exhaustive kernel to within the FP32 charges."""
    wl = synth.config4(0.004)
    q, r = wl.queries, wl.refs
    diam = synth.bbox_diagonal(r)
    h = np.array([0.2, 0.4, 0.8]) * diam
    tq, tr, tw = _dev(q), _dev(r), _dev(wl.weights)
    o = gs.gs_opts_default()
    o.leaf_size = 128
    o.selector = gs.GS_SEL_EXHAUSTIVE
    st = gs.gs_stats()
    got = gs.gs_sum(tq, tr, tw, h, 1e-3, opts=o, stats=st).cpu().numpy()
    assert st.point_pairs_tc == st.point_pairs_base > 0, st.as_dict()
    exact = oracle_ex.gauss_sum(q, r, wl.weights, h)
    err = np.abs(got - exact) / exact
    assert err.max() <= st.fp32_rel_bound, (err.max(), st.fp32_rel_bound)
