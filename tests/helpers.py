"""Shared test helpers: error measures with the library's relative floor."""
import numpy as np


def rel_err(got, want, w_sum=None, floor_log2=-40):
    """|got - want| / max(want, 2^floor_log2 * W) elementwise (the library's
    certified error measure; with w_sum None the floor is 0)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    den = want if w_sum is None else np.maximum(want, 2.0 ** floor_log2 * w_sum)
    return np.abs(got - want) / den
