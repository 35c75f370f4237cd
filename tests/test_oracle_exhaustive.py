"""Pins for the FP64 exhaustive oracle (Section 1's definition of G).

Each check compares the oracle with something the mathematics fixes on its
own: a single term, coincident points, a separable lattice whose sum factors
into 1-D sums, the h -> infinity / h -> 0 limits, and an exactly summable
equal-term case.  A dropped term, a wrong stride or index, a transposed
operand, or a wrong 2 in 2h^2 fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import exhaustive as ex


def test_single_reference_is_one_exponential():
    rng = np.random.default_rng(1)
    for D in (1, 2, 3, 7):
        xq = rng.uniform(0, 1, (5, D))
        xr = rng.uniform(0, 1, (1, D))
        w = np.array([0.37])
        h = np.array([0.05, 0.3, 2.0])
        G = ex.gauss_sum(xq, xr, w, h)
        for q in range(5):
            d2 = sum((xq[q, d] - xr[0, d]) ** 2 for d in range(D))
            for j, hj in enumerate(h):
                arg = d2 / (2 * hj * hj)
                want = 0.37 * math.exp(-arg)
                # an argument rounded at 2^-53 relative moves exp by arg * 2^-53
                assert G[q, j] == pytest.approx(want, rel=(4 + arg) * 2.0 ** -52, abs=0)


def test_coincident_points_sum_to_total_weight():
    rng = np.random.default_rng(2)
    x = np.tile(rng.uniform(0, 1, (1, 4)), (300, 1))
    w = rng.uniform(0.5, 1.5, 300)
    G = ex.gauss_sum(x[:3], x, w, [1e-3, 1.0])
    assert np.allclose(G, math.fsum(w), rtol=1e-14, atol=0)


def test_separable_lattice_factorises_into_1d_sums():
    """Refs on a Cartesian lattice with product weights: the D-dimensional sum
    equals the product over dimensions of 1-D Gaussian sums."""
    rng = np.random.default_rng(3)
    axes = [rng.uniform(0, 1, n) for n in (5, 4, 3)]
    uw = [rng.uniform(0.5, 1.5, n) for n in (5, 4, 3)]
    pts, ws = [], []
    for idx in itertools.product(*[range(len(a)) for a in axes]):
        pts.append([axes[d][i] for d, i in enumerate(idx)])
        ws.append(np.prod([uw[d][i] for d, i in enumerate(idx)]))
    pts, ws = np.array(pts), np.array(ws)
    xq = rng.uniform(0, 1, (7, 3))
    h = np.array([0.04, 0.2, 1.5])
    G = ex.gauss_sum(xq, pts, ws, h)
    for q in range(7):
        for j, hj in enumerate(h):
            want = 1.0
            for d in range(3):
                want *= math.fsum(uw[d][i] * math.exp(-(xq[q, d] - axes[d][i]) ** 2 / (2 * hj * hj))
                                  for i in range(len(axes[d])))
            assert G[q, j] == pytest.approx(want, rel=1e-13)


def test_bandwidth_limits():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (200, 3))
    w = rng.uniform(0.5, 1.5, 200)
    G = ex.gauss_sum(x, x, w, [1e9, 1e-9])
    assert np.allclose(G[:, 0], math.fsum(w), rtol=1e-12)      # h -> inf: every kernel -> 1
    assert np.allclose(G[:, 1], w, rtol=1e-15, atol=0)          # h -> 0: only the self term


def test_skip_self_removes_exactly_the_own_weight():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (150, 2))
    w = rng.uniform(0.5, 1.5, 150)
    h = [0.02, 0.3]
    full = ex.gauss_sum(x, x, w, h)
    loo = ex.gauss_sum(x, x, w, h, skip_self=True)
    assert np.allclose(full - loo, w[:, None], rtol=1e-12, atol=1e-15)


def test_compensated_sum_of_many_equal_terms_is_exact():
    """2^20 identical terms sum to 2^20 times the term, to the last bits."""
    n = 1 << 20
    xr = np.full((n, 1), 0.25)
    w = np.full(n, 0.1)
    G = ex.gauss_sum(np.array([[0.0]]), xr, w, [0.5])
    term = 0.1 * math.exp(-0.0625 / 0.5)
    assert G[0, 0] == pytest.approx(n * term, rel=4e-16)


def test_order_of_queries_and_bandwidths():
    """Row q / column j of the output belongs to query q / bandwidth j."""
    xq = np.array([[0.0], [1.0]])
    xr = np.array([[0.0]])
    G = ex.gauss_sum(xq, xr, [1.0], [1.0, 0.5])
    assert G[0, 0] == 1.0 and G[0, 1] == 1.0
    assert G[1, 0] == pytest.approx(math.exp(-0.5), rel=1e-15)
    assert G[1, 1] == pytest.approx(math.exp(-2.0), rel=1e-15)
