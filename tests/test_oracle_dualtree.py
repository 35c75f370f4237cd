"""Pins for the CPU dual-tree reference (tree, traversal, estimate).

The tree is pinned by its defining invariants and by the 1-D case, where the
partition must be the sorted order; the traversal by exact coverage (every
(query, reference, bandwidth) triple lies in exactly one finished pair), by
the Theorem 2 invariant on the error charged to every query, and by its FP64
estimate against the exhaustive oracle.
"""
import math

import numpy as np
import pytest

from oracle import dualtree as T
from oracle import exhaustive as oracle_ex
from workloads import synth


def test_exp2_f32_error_below_margin():
    """The FP32 exp2 used for the kernel bounds stays within 2^-20 relative
    error of 2^x over its whole domain [-125, 0]."""
    x = np.concatenate([-np.linspace(0, 125, 400001), np.random.default_rng(1).uniform(-125, 0, 100000)])
    x32 = x.astype(np.float32)
    got = T.exp2_f32(x32).astype(np.float64)
    want = np.exp2(x32.astype(np.float64))
    assert np.max(np.abs(got - want) / want) < 2.0 ** -20


def test_kernel_bounds_bracket_exact_values():
    """K(delta_max) lower and K(delta_min) / e^{-delta_min^2/4h^2} upper
    bounds hold against the FP64 box distances for every random pair."""
    import math
    from oracle import series as S
    rng = np.random.default_rng(5)
    for D in (1, 2, 3, 7):
        x = rng.uniform(0, 1, (600, D)).astype(np.float32)
        w = np.ones(600, np.float32)
        t = T.build_tree(x, w, 8)
        pq = rng.integers(0, t.nodes, 3000)
        pr = rng.integers(0, t.nodes, 3000)
        for h in (1e-3, 0.02, 0.3, 5.0):
            c32 = np.full(pq.size, np.float32(1.4426950408889634 / ((2.0 * h) * h)))
            kmax, kmin, e4 = T.kernel_bounds(t, t, pq, pr, c32)
            for i in range(0, 3000, 7):
                dmin, dmax = S.box_distances(t.lo[pq[i]], t.hi[pq[i]], t.lo[pr[i]], t.hi[pr[i]])
                assert kmax[i] <= math.exp(-dmax * dmax / (2 * h * h))
                assert kmin[i] >= math.exp(-dmin * dmin / (2 * h * h))
                assert e4[i] >= math.exp(-dmin * dmin / (4 * h * h))


def test_group_reduce_matches_exact_sums():
    rng = np.random.default_rng(2)
    sizes = [1, 5, 31, 32, 33, 64, 100, 1000]
    vals, gid, pos = [], [], []
    for g, s in enumerate(sizes):
        vals.append(rng.uniform(0, 1, s))
        gid.append(np.full(s, g))
        pos.append(np.arange(s))
    v = np.concatenate(vals)
    got = T.group_reduce(v, np.concatenate(gid), np.concatenate(pos), len(sizes))
    for g, x in enumerate(vals):
        assert got[g] == pytest.approx(math.fsum(x), rel=1e-14)


def _check_tree(x, w, L):
    t = T.build_tree(x, w, L)
    n = x.shape[0]
    assert sorted(t.perm.tolist()) == list(range(n))
    assert -(-n // (1 << t.depth)) <= L and (t.depth == 0 or -(-n // (1 << (t.depth - 1))) > L)
    for k in range(t.depth + 1):
        b = T.level_bounds(n, k)
        for i in range(1 << k):
            node = (1 << k) - 1 + i
            seg = t.perm[b[i]:b[i + 1]]
            assert len(seg) >= 1
            if k == t.depth:
                assert np.all(np.diff(seg) > 0)                   # leaves: ascending original index
            pts = x[seg].astype(np.float64)
            assert np.array_equal(t.lo[node], pts.min(0)) and np.array_equal(t.hi[node], pts.max(0))
            assert t.W[node] == pytest.approx(math.fsum(w[seg].astype(np.float64)), rel=1e-13)
            if k < t.depth:
                s = t.split_dim[node]
                ext = pts.max(0) - pts.min(0)
                assert s == int(np.argmax(ext))
                mid = ((2 * i + 1) * n) // (2 << k)
                left, right = t.perm[b[i]:mid], t.perm[mid:b[i + 1]]
                kl = max((x[j, s], j) for j in left)
                kr = min((x[j, s], j) for j in right)
                assert kl < kr                                    # median split by (coord, index)
    return t


@pytest.mark.parametrize("n,D,L", [(1000, 2, 32), (777, 3, 16), (300, 5, 8), (64, 1, 2), (33, 4, 32)])
def test_tree_invariants(n, D, L):
    x, _, w = synth.small_random(n + D, n, D)
    _check_tree(x, w, L)


def test_tree_fp64_and_ties():
    rng = np.random.default_rng(3)
    x = np.round(rng.uniform(0, 1, (500, 2)), 2)                 # many equal coordinates
    w = rng.uniform(0.5, 1.5, 500).astype(np.float32)
    _check_tree(x, w, 8)


def test_tree_1d_is_the_sorted_order():
    rng = np.random.default_rng(4)
    x = np.round(rng.uniform(0, 1, (513, 1)), 3).astype(np.float32)
    w = np.ones(513, np.float32)
    t = T.build_tree(x, w, 4)
    want = np.lexsort((np.arange(513), x[:, 0]))
    for i in range(1 << t.depth):
        b = T.level_bounds(513, t.depth)
        assert set(t.perm[b[i]:b[i + 1]]) == set(want[b[i]:b[i + 1]])


def _problem(seed, n, D, m=None):
    q, r, w = synth.small_random(seed, n, D, m=m)
    mono = m is None
    return q, r, w, mono


def _trees(q, r, w, mono, L):
    rt = T.build_tree(r, w, L)
    qt = rt if mono else T.build_tree(q, np.ones(q.shape[0], np.float32), L)
    return qt, rt


def _coverage(qt, rt, trav, nh):
    cov = np.zeros((qt.n, rt.n, nh), dtype=np.int32)
    for it in trav.iters:
        for q, r, j, m in zip(it["q"], it["r"], it["j"], it["method"]):
            if m != T.SPLIT:
                cov[qt.begin[q]:qt.end[q], rt.begin[r]:rt.end[r], j] += 1
    return cov


@pytest.mark.parametrize("selector", [T.SEL_RULE, T.SEL_FD_ONLY, T.SEL_EXHAUSTIVE])
def test_traversal_covers_every_triple_exactly_once(selector):
    q, r, w, mono = _problem(21, 600, 2)
    qt, rt = _trees(q, r, w, mono, 16)
    h = np.array([0.005, 0.05, 0.5])
    trav = T.traverse(qt, rt, mono, h, 1e-2, selector=selector, w_max=float(w.max()))
    assert np.all(_coverage(qt, rt, trav, h.size) == 1)


@pytest.mark.parametrize("D,n,m,eps,tokens", [(2, 1500, None, 1e-2, True), (3, 1200, None, 1e-3, True),
                                              (3, 1000, 700, 1e-2, True), (2, 1200, None, 1e-2, False),
                                              (5, 800, None, 1e-2, True)])
def test_estimate_within_eps_and_theorem2_invariant(D, n, m, eps, tokens):
    q, r, w, mono = _problem(30 + D, n, D, m)
    qt, rt = _trees(q, r, w, mono, 16)
    h = synth.log_bandwidths(synth.bbox_diagonal(r), 6, 1e-3, 1.0)
    trav = T.traverse(qt, rt, mono, h, eps, tokens=tokens, w_max=float(w.max()))
    got, charged = T.estimate(qt, rt, q, r, w, h, trav)
    want = oracle_ex.gauss_sum(q, r, w, h)
    floor = 2.0 ** -40 * float(np.sum(w.astype(np.float64)))
    den = np.maximum(want, floor)
    assert np.all(charged <= trav.eps_t * den * (1 + 1e-9))          # Theorem 2 with tokens
    assert np.max(np.abs(got - want) / den) <= trav.eps_t * (1 + 1e-6)
    methods = np.concatenate([it["method"] for it in trav.iters])
    assert (methods == T.FD).any() and (methods == T.BASE).any()


@pytest.mark.parametrize("D,m,tokens", [(2, None, True), (3, None, True), (3, 700, True), (2, None, False)])
def test_best_first_lower_bounds_hold_and_estimate_within_eps(D, m, tokens):
    """Best-first look-ahead: every group's G^min (with the children's lower
    bounds of the largest-gap pairs) is still below the exact sum of every
    query of its node (or the floor / the self term that raised it), and the
    estimate keeps Theorem 2's guarantee."""
    q, r, w, mono = _problem(50 + D, 1200, D, m)
    qt, rt = _trees(q, r, w, mono, 16)
    h = synth.log_bandwidths(synth.bbox_diagonal(r), 6, 1e-3, 1.0)
    eps = 1e-2
    trav = T.traverse(qt, rt, mono, h, eps, tokens=tokens, w_max=float(w.max()), best_first=True)
    assert trav.lookahead > 0
    want = oracle_ex.gauss_sum(q, r, w, h)
    W = float(np.sum(w.astype(np.float64)))
    floorW = 2.0 ** -40 * W
    # exact minimum over the queries of each query node, per bandwidth
    sorted_want = want[qt.perm]
    for it in trav.iters:
        qs, js, G = it["q"], it["j"], it["G"]
        mins = np.array([sorted_want[qt.begin[a]:qt.end[a], b].min() for a, b in zip(qs, js)])
        lower = np.maximum(mins, floorW)
        if mono:
            lower = np.maximum(lower, qt.wmin[qs])
        assert np.all(G <= lower * (1 + 1e-9))
    got, charged = T.estimate(qt, rt, q, r, w, h, trav)
    den = np.maximum(want, floorW)
    assert np.all(charged <= trav.eps_t * den * (1 + 1e-9))
    assert np.max(np.abs(got - want) / den) <= trav.eps_t * (1 + 1e-6)
    # the look-ahead can only raise a pair's lower bound: same first iteration, G^min at least as large
    plain = T.traverse(qt, rt, mono, h, eps, tokens=tokens, w_max=float(w.max()))
    assert np.all(trav.iters[0]["G"] >= plain.iters[0]["G"])


def test_series_methods_are_used_in_low_dimension():
    q, r, w, mono = _problem(40, 3000, 2)
    qt, rt = _trees(q, r, w, mono, 16)
    h = np.array([0.1, 0.3])
    # the paper's unit cost weights favour series actions in 2-D
    trav = T.traverse(qt, rt, mono, h, 1e-3, w_max=float(w.max()), cost_weight=(1, 1, 1, 1))
    methods = np.concatenate([it["method"] for it in trav.iters])
    assert np.isin([T.DH, T.DL, T.H2L], methods).any()
    got, _ = T.estimate(qt, rt, q, r, w, h, trav)
    want = oracle_ex.gauss_sum(q, r, w, h)
    assert np.max(np.abs(got - want) / want) <= 1e-3


def test_directed_fp32_arithmetic_brackets_the_exact_result():
    # rounded-down / -up FP32 sums and products bracket the exact rational
    # result by one FP32 step, including operands of very different size
    from fractions import Fraction
    g = np.random.default_rng(17)
    a = (g.standard_normal(400) * 2.0 ** g.integers(-30, 30, 400)).astype(np.float32)
    b = (g.standard_normal(400) * 2.0 ** g.integers(-30, 30, 400)).astype(np.float32)
    for up in (False, True):
        s = T.f32_add_dir(a, b, up)
        p = T.f32_mul_dir(np.abs(a), np.abs(b), up)
        for i in range(a.size):
            es = Fraction(float(a[i])) + Fraction(float(b[i]))
            ep = Fraction(float(abs(a[i]))) * Fraction(float(abs(b[i])))
            for got, ex in ((s[i], es), (p[i], ep)):
                other = np.nextafter(got, np.float32(-np.inf if up else np.inf))
                if up:
                    assert Fraction(float(got)) >= ex and Fraction(float(other)) < ex
                else:
                    assert Fraction(float(got)) <= ex and Fraction(float(other)) > ex


def test_directed_group_sums_bound_the_exact_sums():
    g = np.random.default_rng(18)
    n = 5000
    gid = np.sort(g.integers(0, 37, n))
    start = np.searchsorted(gid, np.arange(37))
    pos = np.arange(n) - start[gid]
    v = g.uniform(0, 1, n).astype(np.float32)
    lo = T.group_reduce_f32(v, gid, pos, 37, up=False)
    hi = T.group_reduce_f32(v, gid, pos, 37, up=True)
    exact = np.bincount(gid, weights=v.astype(np.float64), minlength=37)
    assert np.all(lo <= exact) and np.all(hi >= exact)
    assert np.all(hi - lo <= 1e-5 * exact + 1e-30)


def _run_then_kahan_f32(terms):
    """The base case's accumulation order: an FP32 running sum over each
    reference leaf (a row of `terms`), then a compensated FP32 sum of the
    leaf sums."""
    s = np.float32(0.0)
    c = np.float32(0.0)
    for row in terms:
        part = np.float32(0.0)
        for v in row:
            part = np.float32(part + v)
        y = np.float32(part - c)
        t = np.float32(s + y)
        c = np.float32(np.float32(t - s) - y)
        s = t
    return float(s)


@pytest.mark.parametrize("run", [16, 64, 128])
def test_summation_charge_covers_adversarial_runs(run):
    """Positive terms built so that every FP32 addition of a leaf run rounds
    up by almost a full unit: the relative error of the run-then-compensated
    sum approaches (run - 1) u, which the charge's run-length term covers —
    and for runs of 128 (leaf size 128) it exceeds 64 u."""
    u = 2.0 ** -24
    rows = []
    for leaf in range(4):
        s = np.float32(1.0 + leaf)
        row = [s]
        for _ in range(run - 1):
            # just above half an ulp of the running sum: rounds up to the next float
            ulp = float(np.spacing(np.float32(s)))
            t = np.float32(ulp * 0.5 * (1.0 + 2.0 ** -8))
            row.append(t)
            s = np.float32(s + t)
        rows.append(row)
    exact = math.fsum(float(v) for row in rows for v in row)
    got = _run_then_kahan_f32(rows)
    rel = abs(got - exact) / exact
    charge = T.fp32_rho(1, 1, 0.0, 1.0, -40, run) - T.fp32_rho(1, 1, 0.0, 1.0, -40, 0) + u
    assert rel <= charge
    if run == 128:
        assert rel > 64.0 * u


@pytest.mark.parametrize("D,n,m,leaf", [(2, 1500, None, 16), (3, 1200, 700, 8), (5, 900, None, 32)])
def test_pairs_per_iteration_within_the_reserved_lists(D, n, m, leaf):
    """Small traversals reserve their work lists once, at the worst case: the
    pairs of iteration t are distinct (query node, reference node, bandwidth)
    triples of levels min(t, depth), at most nh 2^min(t, d_Q) 2^min(t, d_R) of
    them, and each action list holds at most the sum of that over the
    iterations (checked on the CPU traversal, which the GPU one reproduces)."""
    q, r, w, mono = _problem(50 + D, n, D, m)
    qt, rt = _trees(q, r, w, mono, leaf)
    h = synth.log_bandwidths(synth.bbox_diagonal(r), 4, 1e-3, 1.0)
    trav = T.traverse(qt, rt, mono, h, 1e-2, w_max=float(w.max()), cost_weight=(1, 1, 1, 1))
    total, counts = 0, {}
    for t, it in enumerate(trav.iters):
        bound = h.size << (min(t, qt.depth) + min(t, rt.depth))
        trip = set(zip(it["q"].tolist(), it["r"].tolist(), it["j"].tolist()))
        assert len(trip) == len(it["q"]) <= bound
        total += bound
        for mth in (T.DH, T.DL, T.H2L, T.BASE):
            counts[mth] = counts.get(mth, 0) + int(np.sum(it["method"] == mth))
    assert all(c <= total for c in counts.values())
    assert counts[T.BASE] > 0
