"""Search for the bandwidth that minimises the LSCV score.

Section 7 sweeps the bandwidth over fixed multiples of an optimum found by
least-squares cross-validation; this module finds that optimum.  The score is
evaluated by the library (gs_lscv_trees: dual-tree sums at h and sqrt(2) h
on one kd-tree built once, then the score reduction on the GPU); the search
itself is host logic: a log-spaced grid over the bracket, refined around the
grid minimum round after round, several bandwidths per call so that each
traversal carries a batch of them.
"""
from __future__ import annotations

import math

import numpy as np


def search(score_fn, lo: float, hi: float, rounds: int = 5, per_round: int = 8):
    """Minimise score_fn over [lo, hi] (0 < lo < hi) on a log scale.

    score_fn(h) takes an array of bandwidths and returns their scores.  Each
    round evaluates per_round (>= 3) log-spaced points of the current bracket
    and keeps the neighbours of the best one as the next bracket (the edge
    interval when the best is at an edge).  Returns (h_best, score_best,
    history) with history a list of (h array, score array) per round; the
    final bracket is the last two neighbours of h_best."""
    if not (0.0 < lo < hi) or per_round < 3 or rounds < 1:
        raise ValueError("need 0 < lo < hi, per_round >= 3, rounds >= 1")
    history = []
    best_h, best_s = None, math.inf
    a, b = math.log(lo), math.log(hi)
    for _ in range(rounds):
        hs = np.exp(np.linspace(a, b, per_round))
        sc = np.asarray(score_fn(hs), dtype=np.float64)
        history.append((hs, sc))
        k = int(np.argmin(sc))
        if sc[k] < best_s:
            best_h, best_s = float(hs[k]), float(sc[k])
        a = math.log(hs[max(k - 1, 0)])
        b = math.log(hs[min(k + 1, per_round - 1)])
        if b <= a:
            break
    return best_h, best_s, history


def certify(score_err_fn, hs, eps: float, shrink: float = 4.0, steps: int = 2, scores=None):
    """Certify the grid minimiser of scores that are only known to within
    error bounds.

    score_err_fn(hs, eps) returns (scores, bounds) with |score - exact| <=
    bound for every bandwidth of hs (ascending).  The minimiser at grid index
    k is certified against its neighbours at distance m when the bound
    interval of score k lies strictly below those of k - m and k + m (one
    side at a grid edge): for a unimodal exact score the exact minimiser
    then lies in [hs[k - m], hs[k + m]].  Starting from the given eps (or the
    given (scores, bounds) already computed at it), m = 1 is tried first;
    while it fails, the whole grid is re-scored at eps / shrink, up to `steps`
    times, and the smallest certified m over those evaluations is kept.
    Returns a dict: certified (bool), k, m, eps (of the certifying
    evaluation), bracket [lo, hi], score, bound."""
    hs = np.asarray(hs, dtype=np.float64)
    n = hs.size
    best = None
    e_cur = eps
    for step in range(steps + 1):
        if step == 0 and scores is not None:
            sc, er = (np.asarray(v, dtype=np.float64) for v in scores)
        else:
            sc, er = (np.asarray(v, dtype=np.float64) for v in score_err_fn(hs, e_cur))
        k = int(np.argmin(sc))
        top = sc[k] + er[k]
        found = None
        for m in range(1, n):
            left_ok = k - m < 0 or top < sc[k - m] - er[k - m]
            right_ok = k + m >= n or top < sc[k + m] - er[k + m]
            if k - m < 0 and k + m >= n:
                break
            if left_ok and right_ok:
                found = m
                break
        if found is not None and (best is None or found < best["m"]):
            best = {"certified": True, "k": k, "m": found, "eps": e_cur,
                    "bracket": [float(hs[max(k - found, 0)]), float(hs[min(k + found, n - 1)])],
                    "score": float(sc[k]), "bound": float(er[k]), "h": float(hs[k])}
        if best is not None and best["m"] == 1:
            break
        e_cur /= shrink
    if best is None:
        k = int(np.argmin(sc))
        best = {"certified": False, "k": k, "m": None, "eps": e_cur * shrink,
                "bracket": [float(hs[0]), float(hs[-1])], "score": float(sc[k]), "bound": float(er[k]),
                "h": float(hs[k])}
    return best


def minimize(points, weights, eps: float, lo: float, hi: float, rounds: int = 5, per_round: int = 8,
             opts=None, stream=None, stats=None, certify_steps: int = 0):
    """The LSCV-optimal bandwidth of a weighted point set on the GPU.

    points (N x D) and weights (N, float32) are torch CUDA tensors; the tree is
    built once (opts.leaf_size) and every round evaluates per_round
    bandwidths in one call.  Returns (h_best, score_best, err_best, history)
    where err_best bounds |score - exact score| at h_best.  stats (a gs_stats)
    receives the statistics of the last call.

    certify_steps > 0 appends a fifth element, certify()'s record for the
    last round's grid: when the score bounds of the best grid point and its
    neighbours overlap, that grid is re-scored at eps / 4, eps / 16, ... (up
    to certify_steps times) on the same tree until they separate, and if they
    never do, the previous round's (coarser) grid is tried the same way;
    h_best, score_best and err_best then come from the certifying evaluation
    (record key grid_round: the round whose grid was certified)."""
    from . import gs
    tree = gs.Tree(points, weights, opts=opts, stream=stream)
    errs = {}
    cert = None
    try:
        def score_fn(hs):
            s, e = gs.gs_lscv_trees(tree, hs, eps, opts=opts, stream=stream, stats=stats)
            for h, v in zip(hs, e):
                errs[float(h)] = float(v)
            return s
        h, s, hist = search(score_fn, lo, hi, rounds, per_round)
        if certify_steps > 0:
            # the last grid first; if its neighbours are too close for the
            # bounds, the grid of the round before (a wider bracket)
            for back in (1, 2):
                if back > len(hist):
                    break
                hs_g, sc_g = hist[-back]
                er_g = np.array([errs[float(v)] for v in hs_g])
                cert = certify(lambda hs, e: gs.gs_lscv_trees(tree, hs, e, opts=opts, stream=stream, stats=stats),
                               hs_g, eps, steps=certify_steps, scores=(sc_g, er_g))
                cert["grid_round"] = len(hist) - back
                if cert["certified"]:
                    h, s = cert["h"], cert["score"]
                    errs[h] = cert["bound"]
                    break
    finally:
        tree.close()
    if certify_steps > 0:
        return h, s, errs[h], hist, cert
    return h, s, errs[h], hist
