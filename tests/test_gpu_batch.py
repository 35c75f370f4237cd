"""gs_sum_batched: many uneven problems in one call.

Every problem's result is within its eps of the FP64 exhaustive oracle (the
exhaustive ones to 1e-5), a failing problem reports its own status without
stopping the others, and an empty batch is a no-op.
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


def _problems():
    out = []
    # uneven batched KDE problems (the batched workload's generator, scaled down)
    for i in (1, 5, 9, 13):
        wl = synth.config5_problem(i, scale=0.1)
        out.append((wl.queries, wl.refs, wl.weights, wl.h[::2], wl.eps))
    q, r, w = synth.small_random(31, 1500, 4, m=700)
    out.append((q, r, w, np.array([0.05, 0.2]), 1e-2))
    q, r, w = synth.small_random(32, 900, 3)
    out.append((q, q, w, np.array([0.02, 0.3]), 0.0))        # exhaustive
    q, r, w = synth.small_random(33, 1200, 2, dtype=np.float64)
    out.append((q, q, w, np.array([0.01, 0.1]), 1e-3))
    return out


def test_batched_problems_within_eps(gs):
    probs = _problems()
    dev = []
    for q, r, w, h, eps in probs:
        tq = _dev(q)
        tr = tq if q is r else _dev(r)
        dev.append((tq, tr, _dev(w), h, eps))
    st = gs.gs_stats()
    outs, status = gs.gs_sum_batched(dev, nworkers=3, stats=st)
    assert status == [0] * len(probs)
    assert st.ms_total > 0 and st.launches > 0
    for (q, r, w, h, eps), out in zip(probs, outs):
        exact = oracle_ex.gauss_sum(q, r, w, h)
        err = rel_err(out.cpu().numpy(), exact, float(w.astype(np.float64).sum()))
        assert err.max() <= (eps if eps > 0 else 1e-5), (q.shape, eps, err.max())


def test_failing_problem_reports_its_status(gs):
    probs = _problems()[:3]
    dev = []
    for k, (q, r, w, h, eps) in enumerate(probs):
        w = w.copy()
        if k == 1:
            w[3] = -1.0                        # invalid weight in problem 1 only
        tq = _dev(q)
        tr = tq if q is r else _dev(r)
        dev.append((tq, tr, _dev(w), h, eps))
    with pytest.raises(gs.GSError) as ei:
        gs.gs_sum_batched(dev, nworkers=2)
    assert ei.value.code == gs.GS_ERR_WEIGHT and "problem 1" in str(ei.value)
    outs, status = gs.gs_sum_batched(dev, nworkers=2, raise_on_error=False)
    assert status[1] == gs.GS_ERR_WEIGHT and status[0] == 0 and status[2] == 0
    q, r, w, h, eps = probs[0]
    exact = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(outs[0].cpu().numpy(), exact, float(w.astype(np.float64).sum())).max() <= eps


def test_empty_batch(gs):
    outs, status = gs.gs_sum_batched([])
    assert outs == [] and status == []


def test_small_problems_summed_exactly_with_the_flag(gs):
    probs = _problems()[:5]
    dev = []
    for q, r, w, h, eps in probs:
        tq = _dev(q)
        tr = tq if q is r else _dev(r)
        dev.append((tq, tr, _dev(w), h, eps))
    o = gs.gs_opts_default()
    o.flags |= gs.GS_FLAG_SMALL_EXHAUSTIVE
    st = gs.gs_stats()
    outs, status = gs.gs_sum_batched(dev, opts=o, stats=st)
    assert status == [0] * len(probs)
    assert st.pairs_split == 0 and st.pairs_fd == 0          # no traversal ran
    for (q, r, w, h, eps), out in zip(probs, outs):
        assert float(q.shape[0]) * r.shape[0] * len(h) <= gs.GS_SMALL_WORK
        exact = oracle_ex.gauss_sum(q, r, w, h)
        assert rel_err(out.cpu().numpy(), exact, float(w.astype(np.float64).sum())).max() <= 1e-5


def test_grouped_exhaustive_problems(gs):
    """Under GS_FLAG_SMALL_EXHAUSTIVE every small FP32 problem with D <= 8
    goes through the grouped exhaustive path (a few launches for all of
    them): each result within 1e-5 of the oracle, far fewer launches than
    problems, and a bad weight in one problem reported for that problem only."""
    wls = [synth.config5_problem(i, scale=0.03) for i in range(40)]
    dev = [(_dev(wl.queries), None, _dev(wl.weights), wl.h, wl.eps) for wl in wls]
    dev = [(q, q, w, h, eps) for q, _, w, h, eps in dev]
    o = gs.gs_opts_default()
    o.flags = gs.GS_FLAG_SMALL_EXHAUSTIVE
    st = gs.gs_stats()
    outs, status = gs.gs_sum_batched(dev, opts=o, nworkers=4, stats=st)
    assert status == [0] * len(wls)
    assert st.launches <= 4 * 7 * 4, st.launches          # four launches per (dimension, chunk) group
    assert st.point_pairs_base == sum(wl.M * wl.N * wl.h.size for wl in wls)
    for wl, out in zip(wls, outs):
        exact = oracle_ex.gauss_sum(wl.queries, wl.refs, wl.weights, wl.h)
        assert np.max(np.abs(out.cpu().numpy() - exact) / exact) <= 1e-5, wl.name
    w = wls[7].weights.copy()
    w[5] = 0.0
    bad = list(dev)
    bad[7] = (dev[7][0], dev[7][1], _dev(w), wls[7].h, wls[7].eps)
    outs, status = gs.gs_sum_batched(bad, opts=o, nworkers=4, raise_on_error=False)
    assert status[7] == gs.GS_ERR_WEIGHT and all(s == 0 for k, s in enumerate(status) if k != 7)
    with pytest.raises(gs.GSError) as ei:
        gs.gs_sum_batched(bad, opts=o, nworkers=4)
    assert ei.value.code == gs.GS_ERR_WEIGHT and "problem 7" in str(ei.value)


def test_small_work_threshold_depends_on_dimension(gs):
    """GS_FLAG_SMALL_EXHAUSTIVE: a two-dimensional problem above
    GS_SMALL_WORK_D2 takes the dual tree, a three-dimensional one of the same
    size the exhaustive sum (below GS_SMALL_WORK); both within eps."""
    n, nh = 100000, 8
    assert gs.GS_SMALL_WORK_D2 < float(n) * n * nh <= gs.GS_SMALL_WORK
    for D, traversal in ((2, True), (3, False)):
        x, _, w = synth.small_random(70 + D, n, D)
        h = synth.log_bandwidths(synth.bbox_diagonal(x), nh)
        o = gs.gs_opts_default()
        o.flags = gs.GS_FLAG_SMALL_EXHAUSTIVE
        st = gs.gs_stats()
        tx = _dev(x)
        out = gs.gs_sum(tx, tx, _dev(w), h, 1e-2, opts=o, stats=st).cpu().numpy()
        assert (st.pairs_split > 0) == traversal, st.as_dict()
        idx = np.random.default_rng(D).choice(n, 200, replace=False)
        exact = oracle_ex.gauss_sum(x[idx], x, w, h)
        assert rel_err(out[idx], exact, float(w.astype(np.float64).sum())).max() <= 1e-2
