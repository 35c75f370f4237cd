"""GPU dual-tree path against the CPU references.

* tree partitions and the full traversal record (every pair of every
  iteration, with the action and series order taken) are bit-exact against
  oracle.dualtree on the same seeded inputs;
* every result is within eps of the FP64 exhaustive oracle,
  |G~ - G| <= eps * max(G, 2^-40 W), query by query.
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


PAPER = (1.0, 1.0, 1.0, 1.0)          # the paper's unit cost weights


def _opts(gs, leaf=32, selector=0, tokens=True, plimit=0, cw=None):
    o = gs.gs_opts_default()
    o.leaf_size = leaf
    o.selector = selector
    o.no_tokens = 0 if tokens else 1
    o.plimit = plimit
    if cw is not None:
        for k in range(4):
            o.cost_weight[k] = cw[k]
    return o


def _cpu_trace(q, r, w, mono, h, eps, leaf, selector, tokens, plimit, cw, best_first=False):
    rt = T.build_tree(r, w, leaf)
    qt = rt if mono else T.build_tree(q, np.ones(q.shape[0], np.float32), leaf)
    trav = T.traverse(qt, rt, mono, h, eps, plimit=plimit or None, selector=selector, tokens=tokens,
                      w_max=float(w.max()), cost_weight=cw, best_first=best_first)
    rec = []
    for t, it in enumerate(trav.iters):
        code = it["method"] | (it["p"] << 8) | (t << 16)
        rec.append(np.stack([it["q"], it["r"], it["j"], code], axis=1))
    return qt, rt, np.concatenate(rec).astype(np.int64), trav


DEF = T.COST_WEIGHTS
CASES = [
    # seed, n, D, m (None: monochromatic), eps, leaf, selector, tokens, plimit, h, cost weights
    (1, 3000, 2, None, 1e-2, 32, 0, True, 0, [0.003, 0.03, 0.3], PAPER),
    (2, 2500, 3, None, 1e-3, 16, 0, True, 0, [0.01, 0.05, 0.2, 0.8], PAPER),
    (3, 2000, 3, 1500, 1e-2, 32, 0, True, 0, [0.02, 0.2], DEF),
    (4, 1800, 5, None, 1e-2, 16, 0, True, 0, [0.05, 0.3, 1.0], PAPER),
    (5, 2200, 2, None, 1e-2, 8, 2, True, 0, [0.01, 0.1], DEF),
    (6, 2200, 2, None, 1e-2, 32, 0, False, 0, [0.01, 0.1], PAPER),
    (7, 1500, 4, None, 1e-2, 32, 3, True, 0, [0.1], DEF),
    (8, 1200, 7, 900, 1e-2, 16, 0, True, 0, [0.1, 0.5], DEF),
    (9, 2000, 2, None, 1e-3, 32, 0, True, 3, [0.05, 0.2], PAPER),
    (10, 6000, 2, None, 1e-2, 32, 0, True, 0, [0.02, 0.1, 0.4], DEF),
    (11, 4000, 3, None, 1e-4, 32, 0, True, 0, [0.05, 0.3], DEF),
    (12, 1500, 12, 1000, 1e-2, 16, 0, True, 0, [0.3, 1.0], DEF),    # tensor-core base case and its charge
    (13, 5000, 3, None, 1e-2, 64, 0, True, 0, [0.01, 0.05, 0.2], DEF),   # two query slots per lane
    (14, 4000, 5, 3000, 1e-3, 128, 0, True, 0, [0.05, 0.3], DEF),        # four query slots per lane
]


def _bit_exact_case(gs, case, best_first=False):
    seed, n, D, m, eps, leaf, sel, tok, plim, h, cw = case
    q, r, w = synth.small_random(seed, n, D, m=m)
    mono = m is None
    h = np.asarray(h, np.float64)
    tq = _dev(q)
    tr = tq if mono else _dev(r)
    o = _opts(gs, leaf, sel, tok, plim, cw)
    if best_first:
        o.flags = gs.GS_FLAG_BEST_FIRST
    out, trace, qperm, rperm = gs.gs_sum_trace(tq, tr, _dev(w), h, eps, opts=o)
    qt, rt, want, trav = _cpu_trace(q, r, w, mono, h, eps, leaf, sel, tok, plim, cw, best_first)
    if best_first:
        assert trav.lookahead > 0
    assert np.array_equal(rperm.cpu().numpy(), rt.perm)
    assert np.array_equal(qperm.cpu().numpy(), qt.perm)
    got = trace.cpu().numpy().astype(np.int64)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.flatnonzero(np.any(got != want, axis=1))
    assert bad.size == 0, "first mismatch at record %d: gpu %s cpu %s" % (bad[0], got[bad[0]], want[bad[0]])
    exact = oracle_ex.gauss_sum(q, r, w, h)
    err = rel_err(out.cpu().numpy(), exact, float(w.astype(np.float64).sum()))
    assert err.max() <= eps, err.max()
    return out


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d_n%d_d%d" % (c[0], c[1], c[2]))
def test_traversal_bit_exact_and_within_eps(gs, case):
    out = _bit_exact_case(gs, case)
    # the traced call sizes its lists iteration by iteration on the host; a
    # plain call of this size reserves them at their worst case and reads no
    # totals until the end: same decisions, same kernels, so the same sums up
    # to the order of the FP64 atomic additions of the series and base phases
    seed, n, D, m, eps, leaf, sel, tok, plim, h, cw = case
    q, r, w = synth.small_random(seed, n, D, m=m)
    tq = _dev(q)
    plain = gs.gs_sum(tq, tq if m is None else _dev(r), _dev(w), np.asarray(h, np.float64), eps,
                      opts=_opts(gs, leaf, sel, tok, plim, cw)).cpu().numpy()
    traced = out.cpu().numpy()
    assert np.max(np.abs(plain - traced) / traced) <= 1e-12


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in (1, 2, 3, 6, 11)],
                         ids=lambda c: "s%d_n%d_d%d" % (c[0], c[1], c[2]))
def test_best_first_traversal_bit_exact_and_within_eps(gs, case):
    """GS_FLAG_BEST_FIRST: the look-ahead of the largest-gap pairs of every
    group, bit-exact against the CPU traversal with best_first=True."""
    _bit_exact_case(gs, case, best_first=True)


def _check_eps(gs, wl, eps=None, opts=None, sample=None):
    eps = wl.eps if eps is None else eps
    tq = _dev(wl.queries)
    tr = tq if wl.mono else _dev(wl.refs)
    st = gs.gs_stats()
    out = gs.gs_sum(tq, tr, _dev(wl.weights), wl.h, eps, opts=opts, stats=st).cpu().numpy()
    qs, o = wl.queries, out
    if sample is not None:
        idx = np.sort(np.random.default_rng(0).choice(wl.M, sample, replace=False))
        qs, o = wl.queries[idx], out[idx]
    exact = oracle_ex.gauss_sum(qs, wl.refs, wl.weights, wl.h)
    err = rel_err(o, exact, float(wl.weights.astype(np.float64).sum()))
    assert err.max() <= eps, (err.max(), st.as_dict())
    return st


def test_config1_full_size_every_query(gs):
    st = _check_eps(gs, synth.config1())
    assert st.pairs_fd + st.pairs_dh + st.pairs_dl + st.pairs_h2l > 0


def test_config2_scaled_sweep(gs):
    _check_eps(gs, synth.config2(0.02))


def test_merged_and_unmerged_base_case_agree(gs):
    """The bandwidth-merged base case and the per-bandwidth one sum the same
    leaf pairs: results agree to FP32 summation accuracy."""
    wl = synth.config2(0.02)
    tq, tw = _dev(wl.queries), _dev(wl.weights)
    a = gs.gs_sum(tq, tq, tw, wl.h, wl.eps).cpu().numpy()
    o = _opts(gs)
    o.flags = gs.GS_FLAG_NO_MERGE
    b = gs.gs_sum(tq, tq, tw, wl.h, wl.eps, opts=o).cpu().numpy()
    assert np.max(np.abs(a - b) / b) <= 1e-5


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_config3_scaled_series_regime(gs, eps):
    _check_eps(gs, synth.config3(0.02, eps=eps), eps=eps)


def test_config4_scaled_bichromatic_d16(gs):
    _check_eps(gs, synth.config4(0.005))


def test_config5_some_batched_problems(gs):
    for i in range(6):
        _check_eps(gs, synth.config5_problem(i, scale=0.1))


def test_config2_full_size_sampled(gs):
    st = _check_eps(gs, synth.config2(), sample=48)
    assert st.point_pairs_base < 1e12 * 16      # the tree pruned something


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_config3_full_size_sampled(gs, eps):
    # D = 5, 5e5 points, 8 bandwidths: every query of a seeded sample checked
    wl = synth.config3(eps=eps)
    st = _check_eps(gs, wl, eps=eps, sample=64)
    assert st.pairs_fd > 0


def test_config4_full_size_sampled(gs):
    # D = 16 bichromatic: 2e6 references, 2e5 queries, 8 bandwidths
    wl = synth.config4()
    st = _check_eps(gs, wl, sample=32)
    assert st.point_pairs_base <= float(wl.M) * wl.N * wl.h.size


@pytest.mark.parametrize("n,m,D", [(1, 1, 2), (5, 3, 1), (40, 1, 3), (1, 50, 2), (64, 64, 32)])
def test_degenerate_sizes(gs, n, m, D):
    q, r, w = synth.small_random(n * 31 + m, n, D, m=m)
    h = np.array([0.01, 0.2, 3.0])
    out = gs.gs_sum(_dev(q), _dev(r), _dev(w), h, 1e-2, opts=_opts(gs, leaf=2)).cpu().numpy()
    exact = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(out, exact, float(w.astype(np.float64).sum())).max() <= 1e-2


def test_coincident_points(gs):
    x = np.tile(np.array([[0.3, 0.7]], np.float32), (500, 1))
    w = np.full(500, 0.002, np.float32)
    out = gs.gs_sum(_dev(x), _dev(x), _dev(w), [1e-3, 1.0], 1e-2).cpu().numpy()
    assert np.allclose(out, 1.0, rtol=1e-2)


@pytest.mark.parametrize("leaf", [2, 5, 64, 128])
def test_leaf_sizes(gs, leaf):
    q, r, w = synth.small_random(77, 3000, 3)
    h = np.array([0.02, 0.2])
    out = gs.gs_sum(_dev(q), _dev(q), _dev(w), h, 1e-2, opts=_opts(gs, leaf=leaf)).cpu().numpy()
    exact = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(out, exact).max() <= 1e-2


def test_small_initial_capacity_grows(gs):
    """Work lists start tiny and must grow between iterations."""
    q, r, w = synth.small_random(78, 4000, 2)
    h = np.array([0.05, 0.5])
    o = _opts(gs, cw=PAPER)
    o.pair_capacity = 64
    out = gs.gs_sum(_dev(q), _dev(q), _dev(w), h, 1e-3, opts=o).cpu().numpy()
    exact = oracle_ex.gauss_sum(q, r, w, h)
    assert rel_err(out, exact).max() <= 1e-3


@pytest.mark.parametrize("D", [2, 3, 5])
def test_paper_cost_model_within_eps(gs, D):
    """Series-heavy runs (the paper's unit cost weights) stay within eps."""
    q, r, w = synth.small_random(90 + D, 8000, D)
    h = synth.log_bandwidths(synth.bbox_diagonal(r), 6, 1e-2, 1.0)
    for eps in (1e-2, 1e-4):
        st = gs.gs_stats()
        out = gs.gs_sum(_dev(q), _dev(q), _dev(w), h, eps, opts=_opts(gs, cw=PAPER), stats=st).cpu().numpy()
        exact = oracle_ex.gauss_sum(q, r, w, h)
        assert rel_err(out, exact).max() <= eps
        if D <= 3:
            assert st.pairs_dh + st.pairs_dl + st.pairs_h2l > 0


def test_autotuner_picks_a_certified_configuration(gs, tmp_path):
    from paper_1206_6857_gb300 import autotune
    wl = synth.config2(0.02)
    tq, tw = _dev(wl.queries), _dev(wl.weights)
    best, table = autotune.tune(tq, tw, wl.h, wl.eps, fraction=0.5, h_subset=4, leaves=(16, 32))
    assert len(table) == 2 * len(autotune.DEFAULT_COSTS)
    assert best["seconds"] == min(r["seconds"] for r in table)
    out = gs.gs_sum(tq, tq, tw, wl.h, wl.eps, opts=autotune.options(best)).cpu().numpy()
    exact = oracle_ex.gauss_sum(wl.queries, wl.refs, wl.weights, wl.h)
    assert rel_err(out, exact).max() <= wl.eps
    key = autotune.key_for(wl.D, wl.N, wl.h, wl.diameter)
    path = str(tmp_path / "tuned.json")
    autotune.cache(path, key, best)
    assert autotune.cache(path, key) == best


H2L_CASES = [
    # seed, n, h, eps, PLIMIT, the orders that must occur (at least that many actions)
    (33, 3000, [0.05, 0.12, 0.3], 3e-2, 4, {3: 100, 4: 1000}),
    (35, 6000, [0.04, 0.1, 0.25], 1e-2, 6, {4: 1000, 5: 10000, 6: 1000}),
]


@pytest.mark.parametrize("case", H2L_CASES, ids=lambda c: "s%d_P%d" % (c[0], c[4]))
def test_h2l_orders_3_to_5_in_three_dimensions(gs, case):
    """H2L-heavy traversals in D = 3 (cost weights that make H2L the cheapest
    method wherever it is certified): the actions at orders 3 to 5 run in
    their own dimension-by-dimension kernel, the others in the general one.
    Bit-exact decisions, and every query's error stays under the bounds
    charged to it (the sum of E over the approximations that cover it) plus
    the FP32 base-case charge, which is far tighter than eps."""
    seed, n, h, eps, P, orders = case
    q, _, w = synth.small_random(seed, n, 3)
    h = np.asarray(h)
    leaf, cw = 16, (1e6, 1e6, 1e-3, 1.0)
    tq = _dev(q)
    st = gs.gs_stats()
    out, trace, _, _ = gs.gs_sum_trace(tq, tq, _dev(w), h, eps, opts=_opts(gs, leaf, 0, True, P, cw), stats=st)
    qt, rt, want, trav = _cpu_trace(q, q, w, True, h, eps, leaf, 0, True, P, cw)
    got = trace.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want)
    act, p = got[:, 3] & 0xff, (got[:, 3] >> 8) & 0xff
    for order, least in orders.items():
        assert np.sum((act == T.H2L) & (p == order)) >= least, (order, np.bincount(p[act == T.H2L]))
    charged = np.zeros((qt.n, h.size))
    for it in trav.iters:
        for qn, j, m, e in zip(it["q"], it["j"], it["method"], it["E"]):
            if m in (T.FD, T.DH, T.DL, T.H2L):
                charged[qt.begin[qn]:qt.end[qn], j] += e
    bound = np.empty_like(charged)
    bound[qt.perm] = charged
    exact = oracle_ex.gauss_sum(q, q, w, h)
    W = float(w.astype(np.float64).sum())
    err = np.abs(out.cpu().numpy() - exact)
    slack = bound + 2.0 * st.fp32_rel_bound * exact + 1e-12 * W
    assert np.all(err <= slack), np.max(err / slack)
    assert np.max(bound / exact) < eps


def test_more_bandwidths_than_one_mask(gs):
    """40 bandwidths in one traversal: more than the merged base case's 32-bit
    bandwidth mask holds, so the per-bandwidth base case runs; every query
    within eps of the oracle."""
    q, _, w = synth.small_random(79, 3000, 2)
    h = np.geomspace(0.005, 0.5, 40)
    out = gs.gs_sum(_dev(q), _dev(q), _dev(w), h, 1e-2, opts=_opts(gs, leaf=32)).cpu().numpy()
    exact = oracle_ex.gauss_sum(q, q, w, h)
    assert rel_err(out, exact, float(w.astype(np.float64).sum())).max() <= 1e-2
