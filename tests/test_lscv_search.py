"""The bandwidth search of paper_1206_6857_gb300.lscv_search (host logic):
on a closed-form objective it brackets the known minimiser, and on the exact
LSCV score of a small sample (the FP64 oracle as the objective) it finds the
minimiser that a dense brute-force grid finds."""
import math

import numpy as np
import pytest

from oracle import lscv as oracle_lscv
from paper_1206_6857_gb300 import lscv_search


def _final_bracket(history, h_best):
    hs = history[-1][0]
    k = int(np.argmin(np.abs(hs - h_best)))
    return hs[max(k - 1, 0)], hs[min(k + 1, hs.size - 1)]


@pytest.mark.parametrize("h0", [0.0371, 0.2, 0.0011])
def test_search_brackets_a_known_minimum(h0):
    f = lambda hs: (np.log(hs) - math.log(h0)) ** 2 + 3.0
    h, s, hist = lscv_search.search(f, 1e-3, 1.0, rounds=6, per_round=8)
    lo, hi = _final_bracket(hist, h)
    assert lo <= h0 <= hi or abs(math.log(h / h0)) < 1e-9
    assert s == pytest.approx(3.0 + math.log(h / h0) ** 2)
    assert abs(math.log(h / h0)) < 0.02


def test_search_edge_and_arguments():
    h, _, _ = lscv_search.search(lambda hs: hs, 0.1, 1.0)          # increasing: the lower edge
    assert h == pytest.approx(0.1)
    with pytest.raises(ValueError):
        lscv_search.search(lambda hs: hs, 1.0, 0.1)
    with pytest.raises(ValueError):
        lscv_search.search(lambda hs: hs, 0.1, 1.0, per_round=2)


def test_search_on_the_exact_lscv_score():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0.3, 0.05, 150), rng.normal(0.7, 0.08, 150)])[:, None]
    w = np.full(x.shape[0], 1.0, np.float32)
    score = lambda hs: oracle_lscv.lscv(x, w, np.asarray(hs))
    h, s, hist = lscv_search.search(score, 1e-3, 1.0, rounds=6, per_round=8)
    grid = np.geomspace(1e-3, 1.0, 400)
    sg = np.concatenate([score(grid[i:i + 32]) for i in range(0, grid.size, 32)])
    g = grid[int(np.argmin(sg))]
    step = math.log(grid[1] / grid[0])
    assert abs(math.log(h / g)) <= 2 * step
    assert s <= sg.min() + 1e-3 * abs(sg.min())
