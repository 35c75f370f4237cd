"""gs_lscv against the oracle's exact LSCV scores (Section 7's bandwidth
selection criterion)."""
import numpy as np
import pytest

from oracle import lscv as oracle_lscv
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


@pytest.mark.parametrize("D,n", [(2, 3000), (3, 2500), (5, 1500)])
def test_lscv_exhaustive_and_dualtree(gs, D, n):
    x, _, w = synth.small_random(200 + D, n, D)
    h = synth.log_bandwidths(synth.bbox_diagonal(x), 8, 1e-2, 1.0)
    want = oracle_lscv.lscv(x, w, h)
    tx, tw = _dev(x), _dev(w)
    got0, err0 = gs.gs_lscv(tx, tw, h, 0.0)
    # exhaustive mode: every G within 1e-5, so the score within the bound that 1e-5 implies
    _, scale = gs.gs_lscv(tx, tw, h, 1e-2)
    tol0 = scale / 1e-2 * 1e-5
    assert np.all(np.abs(got0 - want) <= tol0 + 1e-12 * np.abs(want))
    for eps in (1e-2, 1e-3):
        got, err = gs.gs_lscv(tx, tw, h, eps)
        assert np.all(np.abs(got - want) <= err * (1 + 1e-6) + tol0)


def test_lscv_full_size_sweep_runs(gs):
    wl = synth.config2(0.05)
    score, err = gs.gs_lscv(_dev(wl.queries), _dev(wl.weights), wl.h, wl.eps)
    assert np.all(np.isfinite(score)) and np.all(err >= 0)
    # the optimum lies strictly inside the sweep for clustered data
    k = int(np.argmin(score))
    assert 0 < k < wl.h.size - 1


def test_lscv_trees_equal_gs_lscv(gs):
    """gs_lscv_trees on a built tree gives gs_lscv's scores."""
    x, _, w = synth.small_random(210, 4000, 3)
    h = synth.log_bandwidths(synth.bbox_diagonal(x), 6, 1e-2, 1.0)
    tx, tw = _dev(x), _dev(w)
    a, ea = gs.gs_lscv(tx, tw, h, 1e-2)
    tree = gs.Tree(tx, tw)
    b, eb = gs.gs_lscv_trees(tree, h, 1e-2)
    tree.close()
    assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(a).max())
    assert np.allclose(ea, eb, rtol=1e-9)


def test_bandwidth_search_matches_the_oracle_search(gs):
    """lscv_search.minimize (GPU scores on one tree) against the same search
    run on the oracle's exact scores: the same bandwidth, or one whose exact
    score is within the GPU score's error bound of the oracle's best."""
    from paper_1206_6857_gb300 import lscv_search
    x, _, w = synth.small_random(211, 3000, 2)
    diam = synth.bbox_diagonal(x)
    lo, hi = 1e-3 * diam, diam
    tx, tw = _dev(x), _dev(w)
    h, s, err, hist = lscv_search.minimize(tx, tw, 1e-3, lo, hi, rounds=4, per_round=8)
    ho, so, _ = lscv_search.search(lambda hs: oracle_lscv.lscv(x, w, np.asarray(hs)), lo, hi, rounds=4, per_round=8)
    exact_at_h = float(oracle_lscv.lscv(x, w, np.array([h]))[0])
    assert abs(s - exact_at_h) <= err * (1 + 1e-6)
    assert h == pytest.approx(ho, rel=1e-12) or exact_at_h <= so + 2 * err
    assert sum(len(hs) for hs, _ in hist) == 32


def test_certified_search_brackets_the_exact_grid_minimiser(gs):
    """With certification, the reported bracket of the last grid contains
    the grid point where the oracle's exact score is smallest, and the
    reported score is within its bound of the exact score."""
    from paper_1206_6857_gb300 import lscv_search
    x, _, w = synth.small_random(212, 4000, 3)
    diam = synth.bbox_diagonal(x)
    tx, tw = _dev(x), _dev(w)
    h, s, err, hist, cert = lscv_search.minimize(tx, tw, 1e-2, 1e-3 * diam, diam, rounds=3, per_round=8,
                                                 certify_steps=3)
    hs_last = hist[-1][0]
    exact = oracle_lscv.lscv(x, w, hs_last)
    k_exact = int(np.argmin(exact))
    assert abs(s - float(oracle_lscv.lscv(x, w, np.array([h]))[0])) <= err * (1 + 1e-6)
    if cert["certified"]:
        lo, hi = cert["bracket"]
        assert lo <= hs_last[k_exact] <= hi
        assert cert["eps"] <= 1e-2
