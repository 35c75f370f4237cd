"""Pins for the LSCV oracle: a two-point closed form and a 1-D case whose
integral is done by numerical quadrature rather than the Gaussian convolution
identity the oracle relies on."""
import math

import numpy as np
import pytest

from oracle import lscv as L


def test_two_point_closed_form():
    for D in (1, 2, 3):
        x = np.zeros((2, D))
        x[1, 0] = 0.3
        d = 0.3
        for h in (0.05, 0.2, 1.0):
            got = L.lscv(x, np.array([1.0, 1.0]), [h])[0]
            want = (0.5 * (4 * math.pi * h * h) ** (-D / 2) * (1 + math.exp(-d * d / (4 * h * h)))
                    - 2 * (2 * math.pi * h * h) ** (-D / 2) * math.exp(-d * d / (2 * h * h)))
            assert got == pytest.approx(want, rel=1e-12)


def test_one_dimensional_lscv_by_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, 9)
    w = rng.uniform(0.5, 1.5, 9)
    W = w.sum()
    for h in (0.03, 0.1, 0.4):
        def pdf(u, c):
            return math.exp(-(u - c) ** 2 / (2 * h * h)) / math.sqrt(2 * math.pi * h * h)

        def f(u):
            return sum(w[r] * pdf(u, x[r]) for r in range(9)) / W

        brk = sorted(x.tolist())
        int_f2 = integrate.quad(lambda u: f(u) ** 2, -1 - 10 * h, 2 + 10 * h, points=brk,
                                limit=400, epsabs=1e-13, epsrel=1e-12)[0]
        loo = sum(w[i] / W * sum(w[r] * pdf(x[i], x[r]) for r in range(9) if r != i) / (W - w[i])
                  for i in range(9))
        want = int_f2 - 2 * loo
        assert L.lscv(x, w, [h])[0] == pytest.approx(want, rel=1e-8)


def test_uniform_weights_reduce_to_textbook_score():
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (30, 2))
    n, D, h = 30, 2, 0.15
    got = L.lscv(x, np.full(n, 1.0 / n), [h])[0]
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    t1 = np.exp(-d2 / (4 * h * h)).sum() / (n * n) * (4 * math.pi * h * h) ** (-D / 2)
    off = np.exp(-d2 / (2 * h * h))
    np.fill_diagonal(off, 0)
    t2 = 2 * off.sum() / (n * (n - 1)) * (2 * math.pi * h * h) ** (-D / 2)
    assert got == pytest.approx(t1 - t2, rel=1e-12)
