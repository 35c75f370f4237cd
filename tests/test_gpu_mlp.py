"""Pair-selector network kernels and the learned ordering in the traversal.

* gs_mlp_forward is bit-exact against the FP32 restatement in oracle.mlp;
* gs_mlp_loss_grad matches the FP64 oracle loss and gradient;
* gs_mlp_train fits a learnable labelling;
* GS_SEL_MLP traversals are bit-exact against oracle.dualtree with the same
  network, and every result is within eps of the exhaustive oracle;
* gs_selector_samples gives labelled samples and a cheapest-policy cost no
  larger than the FD-only policy it explored.
"""
import numpy as np
import pytest

from helpers import rel_err
from oracle import dualtree as T
from oracle import exhaustive as oracle_ex
from oracle import mlp
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


def _net(seed):
    # random network whose normalisation puts the features near unit scale
    mu = np.array([-8, -30, 5, 5, 4, -2, 0, 0, -10, 6, 5, 5], np.float64)
    sc = np.full(12, 1.0 / 8.0)
    blob = mlp.init(seed, mu=mu, sc=sc)
    mlp.unpack(blob)["b3"][:] = [0.0, 1.5, 1.5, 1.5, 0.0]   # lean towards the series actions
    return blob


def test_forward_bit_exact(gs):
    g = np.random.default_rng(1)
    blob = mlp.init(3, mu=g.normal(0, 1, 12), sc=g.uniform(0.2, 2.0, 12))
    x = g.normal(0, 3, (1000, 12)).astype(np.float32)
    got = gs.gs_mlp_forward(_dev(blob), _dev(x)).cpu().numpy()
    want = mlp.infer_f32(blob, x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_loss_and_gradient_match_fp64_oracle(gs):
    g = np.random.default_rng(2)
    blob = mlp.init(4, mu=g.normal(0, 0.5, 12), sc=g.uniform(0.5, 1.5, 12))
    p = mlp.unpack(blob)
    p["b1"][:] = g.normal(0, 0.1, 64)
    p["b2"][:] = g.normal(0, 0.1, 64)
    n = 700   # several tiles of 128 and a ragged tail
    x = g.normal(0, 1, (n, 12)).astype(np.float32)
    y = g.integers(0, 5, n).astype(np.int32)
    s = g.uniform(0.5, 2.0, n).astype(np.float32)
    loss, grad = gs.gs_mlp_loss_grad(_dev(blob), _dev(x), _dev(y), _dev(s))
    want_l = mlp.loss(blob.astype(np.float64), x.astype(np.float64), y, s.astype(np.float64))
    want_g = mlp.grad(blob.astype(np.float64), x.astype(np.float64), y, s.astype(np.float64))
    assert float(loss.cpu()) == pytest.approx(want_l, rel=1e-5)
    got = grad.cpu().numpy()
    scale = np.abs(want_g).max()
    assert np.all(np.abs(got - want_g) <= 2e-5 * scale + 1e-4 * np.abs(want_g)), np.abs(got - want_g).max() / scale
    assert not got[:24].any()


def test_training_fits_a_learnable_labelling(gs):
    import torch
    g = np.random.default_rng(5)
    n = 20000
    x = g.normal(0, 1, (n, 12)).astype(np.float32) * 3 + 1
    A = g.normal(0, 1, (12, 5))
    y = np.argmax((x - 1) @ A, axis=1).astype(np.int32)
    params = _dev(mlp.init(6))
    losses = gs.gs_mlp_train(params, _dev(x), _dev(y), None, epochs=25, batch=512, lr=3e-3, seed=7, set_norm=True)
    assert losses[-1] < 0.5 * losses[0]
    pr = mlp.unpack(params.cpu().numpy())
    assert np.allclose(pr["mu"], x.mean(axis=0), atol=1e-3, rtol=1e-4)
    scores = gs.gs_mlp_forward(params, _dev(x)).cpu().numpy()
    acc = float(np.mean(scores.argmax(axis=1) == y))
    assert acc > 0.9, acc


CASES = [
    # seed, n, D, m, eps, leaf, tokens, h, network seed, pairs the network must score
    (21, 3000, 2, None, 1e-2, 32, True, [0.003, 0.03, 0.3], 1, 1),
    (22, 2500, 3, None, 1e-3, 16, True, [0.01, 0.05, 0.2, 0.8], 2, 1),
    (23, 2000, 3, 1500, 1e-2, 32, True, [0.02, 0.2], 3, 0),
    (24, 1800, 5, None, 1e-2, 16, False, [0.05, 0.3, 1.0], 4, 0),
    (25, 4000, 2, None, 1e-4, 32, True, [0.05, 0.3], 5, 0),
    (26, 8000, 2, None, 1e-2, 32, True, [0.1, 0.3, 1.0], 6, 20),
    (27, 6000, 3, None, 1e-2, 32, True, [0.2, 0.5, 1.0], 7, 10),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_n%d_d%d" % (c[0], c[1], c[2]))
def test_learned_ordering_bit_exact_and_within_eps(gs, case):
    seed, n, D, m, eps, leaf, tok, h, nseed, min_consulted = case
    q, r, w = synth.small_random(seed, n, D, m=m)
    mono = m is None
    h = np.asarray(h, np.float64)
    blob = _net(nseed)
    params = _dev(blob)
    o = gs.gs_opts_default()
    o.leaf_size = leaf
    o.no_tokens = 0 if tok else 1
    o.selector = gs.GS_SEL_MLP
    o.selector_params = params.data_ptr()
    tq = _dev(q)
    tr = tq if mono else _dev(r)
    out, trace, qperm, rperm = gs.gs_sum_trace(tq, tr, _dev(w), h, eps, opts=o)
    rt = T.build_tree(r, w, leaf)
    qt = rt if mono else T.build_tree(q, np.ones(q.shape[0], np.float32), leaf)
    trav = T.traverse(qt, rt, mono, h, eps, selector=T.SEL_MLP, tokens=tok, w_max=float(w.max()),
                      mlp_params=blob)
    want = np.concatenate([np.stack([it["q"], it["r"], it["j"], it["method"] | (it["p"] << 8) | (t << 16)], axis=1)
                           for t, it in enumerate(trav.iters)]).astype(np.int64)
    got = trace.cpu().numpy().astype(np.int64)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.flatnonzero(np.any(got != want, axis=1))
    assert bad.size == 0, "first mismatch at record %d: gpu %s cpu %s" % (bad[0], got[bad[0]], want[bad[0]])
    assert trav.consulted >= min_consulted
    exact = oracle_ex.gauss_sum(q, r, w, h)
    err = rel_err(out.cpu().numpy(), exact, float(w.astype(np.float64).sum()))
    assert err.max() <= eps, err.max()


def test_mlp_selector_needs_parameters(gs):
    q, r, w = synth.small_random(1, 500, 2)
    o = gs.gs_opts_default()
    o.selector = gs.GS_SEL_MLP
    with pytest.raises(gs.GSError) as ei:
        gs.gs_sum(_dev(q), _dev(q), _dev(w), [0.1], 1e-2, opts=o)
    assert ei.value.code == gs.GS_ERR_ARG


def test_selector_samples(gs):
    from paper_1206_6857_gb300 import selector
    wl = synth.config2(scale=0.03)
    p = _dev(wl.refs)
    o = gs.gs_opts_default()
    x, y, s, mc = selector.samples(p, _dev(wl.weights), wl.h, wl.eps, opts=o)
    x, y, s = x.cpu().numpy(), y.cpu().numpy(), s.cpu().numpy()
    assert x.shape[0] > 10 and x.shape == (y.size, 12)
    assert np.isfinite(x).all() and set(np.unique(y)) <= {1, 2, 3, 4}
    assert (s >= 0).all() and abs(float(s.mean()) - 1.0) < 1e-3
    assert np.all(x[:, 4] == 3) and np.all(x[:, 1] <= x[:, 0])   # D; K(dmax) <= K(dmin)
    assert 0 < mc[0] <= mc[1] * (1 + 1e-12)
    # the sample count is reported even when the capacity is too small
    with pytest.raises(gs.GSError) as ei:
        gs.gs_selector_samples(p, p, _dev(wl.weights), wl.h, wl.eps, selector.UNIT_COSTS, 10, opts=o)
    assert ei.value.code == gs.GS_ERR_CAPACITY


def test_trained_selector_against_the_rule(gs, capsys):
    """The stored network (trained on the GPU by selector.main) on problems it
    was not trained on: both orderings stay within eps of the oracle; the
    test reports the wall time of each (the gain or loss of the network) and
    fails if the network falls below x0.75 of the rule."""
    import time
    import torch
    from paper_1206_6857_gb300 import selector
    params = selector.load()
    rows = []
    for wl in (synth.config2(scale=0.05), synth.config5_problem(3, scale=0.5)):
        p = _dev(wl.refs)
        w = _dev(wl.weights)
        res = {}
        for name in ("rule", "mlp"):
            o = gs.gs_opts_default()
            o.leaf_size = wl.leaf_size
            if name == "mlp":
                o = selector.options(params, o)
            gs.gs_sum(p, p, w, wl.h, wl.eps, opts=o)
            torch.cuda.synchronize()
            best = None
            for _ in range(3):
                st = gs.gs_stats()
                t0 = time.perf_counter()
                out = gs.gs_sum(p, p, w, wl.h, wl.eps, opts=o, stats=st)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            idx = np.sort(np.random.default_rng(0).choice(wl.M, 300, replace=False))
            exact = oracle_ex.gauss_sum(wl.queries[idx], wl.refs, wl.weights, wl.h)
            err = rel_err(out.cpu().numpy()[idx], exact, float(wl.weights.astype(np.float64).sum()))
            assert err.max() <= wl.eps, (wl.name, name, err.max())
            res[name] = (best, st.pairs_dh + st.pairs_dl + st.pairs_h2l, st.pairs_base)
        assert res["mlp"][1:] != res["rule"][1:]       # the network changed decisions
        ratio = res["rule"][0] / res["mlp"][0]
        rows.append("%s: rule %.2f ms, learned %.2f ms (x%.2f)" % (wl.name, 1e3 * res["rule"][0],
                                                                 1e3 * res["mlp"][0], ratio))
        # the stored network is measured at x0.86 and x0.99 of the rule on these
        # two problems (its series actions at large nodes cost more than its
        # labels model); a drop below x0.75 is a regression of the selector or
        # the series kernels
        assert ratio >= 0.75, rows[-1]
    with capsys.disabled():
        print("\n" + "\n".join(rows))
