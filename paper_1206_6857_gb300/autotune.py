"""Autotuner for the dual-tree parameters the paper fixes by hand.

Section 6 fixes the leaf threshold and PLIMIT per dimension and notes that
the cost cutoffs of bestMethod could be hand-tuned.  On a GPU the relative
cost of an FP64 series action and an FP32 base-case term depends on the
kernels, so this module picks, per workload, the leaf size L, the highest
series order P and the bestMethod cost weights by timing the library itself
on a seeded subsample of the caller's data (same dimension, bandwidths and
eps).  Every candidate is a certified configuration: the choice only moves
time, never the eps guarantee.

The result is a plain dict of gs_opts fields; `cache` persists it as JSON
keyed by (D, N bucket, bandwidth range) so a later run can skip the search.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time

import numpy as np

from . import gs

DEFAULT_LEAVES = (32, 64, 128)
DEFAULT_COSTS = ((32.0, 32.0, 32.0, 1.0), (128.0, 128.0, 4.0, 1.0), (256.0, 256.0, 0.5, 1.0),
                 (256.0, 256.0, 1.0, 1.0), (256.0, 256.0, 2.0, 1.0), (256.0, 256.0, 4.0, 1.0),
                 (512.0, 512.0, 1.0, 1.0), (512.0, 512.0, 2.0, 1.0), (2048.0, 2048.0, 256.0, 1.0))


def key_for(D, N, h, diameter):
    nb = int(round(math.log10(max(N, 1))))
    lo = int(math.floor(math.log10(min(h) / diameter)))
    hi = int(math.ceil(math.log10(max(h) / diameter)))
    return "D%d_N1e%d_h%d..%d" % (D, nb, lo, hi)


def _opts(leaf, plimit, cw):
    o = gs.gs_opts_default()
    o.leaf_size = int(leaf)
    o.plimit = int(plimit)
    for k in range(4):
        o.cost_weight[k] = float(cw[k])
    return o


def default_plimits(D):
    """PLIMIT candidates: the Section 6 table (0) and, where series orders
    are affordable (D <= 8), every even order from 2 to 8."""
    return (0, 2, 4, 6, 8) if D <= 8 else (0,)


def tune(points, weights, h, eps, fraction=1.0, h_subset=8, leaves=DEFAULT_LEAVES, costs=DEFAULT_COSTS,
         plimits=(0,), seed=0, reps=1, queries=None):
    """Time every candidate on a seeded subsample; returns (best dict, table).

    points, weights (and queries for a bichromatic problem) are torch CUDA
    tensors; h is a host sequence.  The timing problem keeps a fraction of the
    points (all by default: point density decides how deep the traversal
    goes, so a thinned sample would favour the wrong settings) and h_subset
    bandwidths spread evenly over h (bandwidths are summed independently, so a
    spread subset predicts the full sweep's balance)."""
    import torch
    h = np.asarray(h, dtype=np.float64)
    if h_subset and h.size > h_subset:
        h = np.sort(h)[np.linspace(0, h.size - 1, h_subset).round().astype(int)]
    N = points.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = max(2, int(N * fraction))
    idx = torch.randperm(N, generator=g)[:n].to(points.device)
    sub_p = points.index_select(0, idx).contiguous()
    sub_w = weights.index_select(0, idx).contiguous()
    if queries is None:
        sub_q = sub_p
    else:
        M = queries.shape[0]
        m = max(1, int(M * fraction))
        qi = torch.randperm(M, generator=g)[:m].to(points.device)
        sub_q = queries.index_select(0, qi).contiguous()
    out = torch.empty((sub_q.shape[0], len(h)), dtype=torch.float64, device=points.device)
    table = []
    for leaf, cw, P in itertools.product(leaves, costs, plimits):
        o = _opts(leaf, P, cw)
        try:
            gs.gs_sum(sub_q, sub_p, sub_w, h, eps, out=out, opts=o)          # warm
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                gs.gs_sum(sub_q, sub_p, sub_w, h, eps, out=out, opts=o)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
        except gs.GSError as err:
            # a candidate whose work lists do not fit the device is not a
            # configuration this problem can use: record it and go on
            if err.code != gs.GS_ERR_OOM:
                raise
            gs.gs_trim_memory(0)
            table.append({"leaf_size": leaf, "plimit": P, "cost_weight": list(cw), "seconds": float("inf"),
                          "out_of_memory": True})
            continue
        table.append({"leaf_size": leaf, "plimit": P, "cost_weight": list(cw), "seconds": float(min(ts))})
    if all(r["seconds"] == float("inf") for r in table):
        raise gs.GSError(gs.GS_ERR_OOM, "every autotuner candidate ran out of device memory")
    best = min(table, key=lambda r: r["seconds"])
    return best, table


def tune_staged(points, weights, h, eps, D, queries=None, **kw):
    """tune() over leaf sizes and cost weights at the Section 6 PLIMIT, then
    over PLIMIT (default_plimits(D)) at the best leaf size and weights: the
    series order only matters where series actions are chosen, so the second
    stage is a short one.  Returns (best, table of both stages)."""
    best, table = tune(points, weights, h, eps, queries=queries, **kw)
    extra = [P for P in default_plimits(D) if P != 0]
    if extra:
        kw2 = dict(kw)
        kw2.update(leaves=(best["leaf_size"],), costs=(tuple(best["cost_weight"]),), plimits=tuple(extra))
        b2, t2 = tune(points, weights, h, eps, queries=queries, **kw2)
        table = table + t2
        if b2["seconds"] < best["seconds"]:
            best = b2
    return best, table


def options(best: dict):
    """gs_opts built from a tuned dict."""
    return _opts(best["leaf_size"], best["plimit"], best["cost_weight"])


def cache(path, key, best=None):
    """Read (best=None) or write the tuned entry for key in a JSON file."""
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    if best is None:
        return data.get(key)
    data[key] = best
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return best
