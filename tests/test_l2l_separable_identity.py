"""Lemma 3's local-to-local shift factorises over the dimensions: the
multinomial coefficient beta! / (alpha! (beta - alpha)!) is a product of
1-D binomials and the power a product of 1-D powers, so the shift can be
applied one dimension at a time (each 1-D shift only lowers that index, so
the total-degree truncation |beta| < p is kept).  Checked on the CPU against
the oracle's direct double sum, D = 1..4, orders 1..6 -- the form a
dimension-by-dimension downward-pass kernel would use."""
import math

import numpy as np
import pytest

from oracle import series as S


def _l2l_by_dimension(B, x_Qp, x_Q, h, p, D):
    s = math.sqrt(2.0 * h * h)
    delta = (np.asarray(x_Q, np.float64) - x_Qp) / s
    al = [tuple(a) for a in S.multi_indices(D, p)]
    cur = {a: float(B[i]) for i, a in enumerate(al)}
    for d in range(D):
        nxt = {}
        for a in al:
            acc = 0.0
            for k in range(a[d], p - (sum(a) - a[d])):
                b = a[:d] + (k,) + a[d + 1:]
                acc += math.comb(k, a[d]) * cur[b] * delta[d] ** (k - a[d])
            nxt[a] = acc
        cur = nxt
    return np.array([cur[a] for a in al])


@pytest.mark.parametrize("D,p", [(1, 6), (2, 5), (3, 3), (3, 6), (4, 4)])
def test_shift_by_dimension_equals_lemma3(D, p):
    rng = np.random.default_rng(10 * D + p)
    B = rng.standard_normal(S.num_terms(D, p))
    x_Qp = rng.uniform(0, 1, D)
    x_Q = x_Qp + rng.normal(0, 0.2, D)
    h = rng.uniform(0.1, 0.5)
    want = S.l2l(B, x_Qp, x_Q, h, p)
    got = _l2l_by_dimension(B, x_Qp, x_Q, h, p, D)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
