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


def minimize(points, weights, eps: float, lo: float, hi: float, rounds: int = 5, per_round: int = 8,
             opts=None, stream=None, stats=None):
    """The LSCV-optimal bandwidth of a weighted point set on the GPU.

    points (N x D) and weights (N, float32) are torch CUDA tensors; the tree is
    built once (opts.leaf_size) and every round evaluates per_round
    bandwidths in one call.  Returns (h_best, score_best, err_best, history)
    where err_best bounds |score - exact score| at h_best.  stats (a gs_stats)
    receives the statistics of the last call."""
    from . import gs
    tree = gs.Tree(points, weights, opts=opts, stream=stream)
    errs = {}
    try:
        def score_fn(hs):
            s, e = gs.gs_lscv_trees(tree, hs, eps, opts=opts, stream=stream, stats=stats)
            for h, v in zip(hs, e):
                errs[float(h)] = float(v)
            return s
        h, s, hist = search(score_fn, lo, hi, rounds, per_round)
    finally:
        tree.close()
    return h, s, errs[h], hist
