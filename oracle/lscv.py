"""Least-squares cross-validation score from exact FP64 sums.

TEST INFRASTRUCTURE ONLY.  Section 7 selects bandwidths by the standard
least-squares cross-validation score (Silverman 1986); the paper does not print
the formula, so this is the textbook score written for a weighted Gaussian
kernel density estimate with normalised weights wbar_i = w_i / W:

  f(x)      = sum_r wbar_r phi_h(x - x_r),  phi_h(u) = (2 pi h^2)^{-D/2} e^{-|u|^2/2h^2}
  f_{-i}(x) = sum_{r != i} w_r phi_h(x - x_r) / (W - w_i)
  LSCV(h)   = int f^2 - 2 sum_i wbar_i f_{-i}(x_i)

With the Gaussian convolution identity int phi_h(x-a) phi_h(x-b) dx =
phi_{sqrt2 h}(a-b) both parts are Gaussian sums over the data itself:
  int f^2 = (4 pi h^2)^{-D/2} sum_i wbar_i G_{sqrt2 h}(x_i) / W
  f_{-i}(x_i) = (2 pi h^2)^{-D/2} (G_h(x_i) - w_i) / (W - w_i).
For w_r = 1/N this is the usual (1/N^2) double sum minus 2/(N(N-1)) times the
leave-one-out sum.
"""
import math

import numpy as np

from . import exhaustive


def lscv_from_sums(w, G_h, G_s2h, h, D):
    """LSCV(h) given G_h(x_i) and G_{sqrt2 h}(x_i) at the data points."""
    w = np.asarray(w, np.float64)
    W = float(np.sum(w))
    wbar = w / W
    term1 = (4 * math.pi * h * h) ** (-D / 2) * float(np.sum(wbar * G_s2h)) / W
    loo = (2 * math.pi * h * h) ** (-D / 2) * (G_h - w) / (W - w)
    term2 = 2.0 * float(np.sum(wbar * loo))
    return term1 - term2


def lscv(x, w, h_list):
    """Exact LSCV scores for every bandwidth in h_list (monochromatic data x)."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    h = np.asarray(h_list, np.float64)
    G = exhaustive.gauss_sum(x, x, w, np.concatenate([h, h * math.sqrt(2.0)]))
    nh = h.size
    return np.array([lscv_from_sums(w, G[:, j], G[:, nh + j], h[j], x.shape[1]) for j in range(nh)])
