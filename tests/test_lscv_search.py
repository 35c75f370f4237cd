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


def _noisy(h0, noise_scale, seed=0):
    """Scores of a log-quadratic with a minimum at h0 plus deterministic
    noise inside a bound proportional to eps (a stand-in for the library's
    eps-implied score bounds)."""
    rng = np.random.default_rng(seed)

    def fn(hs, eps):
        hs = np.asarray(hs)
        exact = (np.log(hs) - math.log(h0)) ** 2
        bound = np.full(hs.size, noise_scale * eps)
        return exact + bound * rng.uniform(-1, 1, hs.size), bound
    return fn


def test_certify_brackets_the_exact_minimiser():
    h0 = 0.0123
    hs = np.geomspace(0.01, 0.016, 8)
    fn = _noisy(h0, 1.0)
    cert = lscv_search.certify(fn, hs, 1e-2, steps=4)
    assert cert["certified"]
    lo, hi = cert["bracket"]
    assert lo <= h0 <= hi
    # the scores separate only once eps is small: the bound shrank with it
    assert cert["eps"] < 1e-2 and cert["bound"] == pytest.approx(1.0 * cert["eps"])


def test_certify_reports_failure_when_bounds_never_separate():
    hs = np.geomspace(0.5, 0.5001, 5)      # a flat stretch: neighbours differ by ~1e-8
    cert = lscv_search.certify(_noisy(0.5, 1.0), hs, 1e-2, steps=1)
    assert not cert["certified"] and cert["m"] is None


def test_certify_edge_minimum_is_one_sided():
    hs = np.geomspace(0.1, 1.0, 6)
    fn = lambda h, e: (np.asarray(h) * 10.0, np.full(len(h), 1e-3))      # increasing: the lower edge
    cert = lscv_search.certify(fn, hs, 1e-2)
    assert cert["certified"] and cert["k"] == 0 and cert["m"] == 1
    assert cert["bracket"] == [pytest.approx(0.1), pytest.approx(hs[1])]
