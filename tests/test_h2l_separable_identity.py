"""The three-dimensional H2L kernel sums Lemma 1's double sum one dimension
at a time (X1 over alpha_3, X2 over alpha_2, then alpha_1, every range cut to
total degree < p).  This checks that reordering on the CPU: the staged sum,
written here in plain numpy, equals the oracle's direct Lemma 1 sum for
random coefficients at orders 1 to 6."""
import math

import numpy as np
import pytest

from oracle import series as S


def _separable_h2l(A, x_R, x_Q, h, p):
    s = math.sqrt(2.0 * h * h)
    tau = (np.asarray(x_Q, np.float64) - x_R) / s
    al = S.multi_indices(3, p)
    pos = {tuple(a): i for i, a in enumerate(al)}
    H = S.hermite_polys(tau, 2 * p - 2)               # (2p-1, 3)
    et = math.exp(-float(tau @ tau))
    C = {}
    for a1 in range(p):
        X1 = {}
        for a2 in range(p - a1):
            for b3 in range(p):
                X1[a2, b3] = sum(A[pos[(a1, a2, a3)]] * H[a3 + b3, 2] for a3 in range(p - a1 - a2))
        for c2 in range(p):
            for c3 in range(p - c2):
                x2 = sum(X1[a2, c3] * H[a2 + c2, 1] for a2 in range(p - a1))
                for c1 in range(p - c2 - c3):
                    C[c1, c2, c3] = C.get((c1, c2, c3), 0.0) + x2 * H[a1 + c1, 0]
    out = np.zeros(len(al))
    for b in al:
        sign = -1.0 if sum(b) % 2 else 1.0
        out[pos[tuple(b)]] = sign / S.mfact(b) * et * C[tuple(b)]
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_staged_sum_equals_lemma1(p):
    rng = np.random.default_rng(100 + p)
    for _ in range(3):
        A = rng.standard_normal(S.num_terms(3, p))
        x_R = rng.uniform(0, 1, 3)
        x_Q = x_R + rng.normal(0, 0.3, 3)
        h = rng.uniform(0.1, 0.5)
        want = S.h2l(A, x_R, x_Q, h, p, p)
        got = _separable_h2l(A, x_R, x_Q, h, p)
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12 * scale)
