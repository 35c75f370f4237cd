"""FP64 reference for the O(D^p) Hermite / Taylor series algebra.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, written from
the paper's definitions in the paper's order; nothing here is blocked, fused or
reordered.  Notation: s = sqrt(2 h^2); "order p" keeps the multi-indices with
|alpha| < p (Section 2: C(D+p-1, D) terms; D=2, p=2 gives 3).

Readings taken where the paper is silent or garbled:
  * graded lexicographic order: |alpha| ascending; inside one degree,
    lexicographically descending in (alpha_1, ..., alpha_D), so degree 1 is
    e_1, e_2, ..., e_D as in the Section 2 worked example;
  * the sign in Lemma 1 is (-1)^{|beta|} (as in Lemmas 5 and 6);
  * the Hermite-function bound used by Lemmas 4-6 is Cramer's inequality
    |h_n(t)| <= 2^{n/2} sqrt(n!) e^{-t^2/2} with constant 1.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


# --------------------------------------------------------------------------
# Multi-index notation (Section 1, footnote 1; Section 2)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def multi_indices(D: int, p: int) -> tuple:
    """All alpha in N^D with |alpha| < p, graded lexicographic order."""
    out = []
    for deg in range(p):
        layer = []

        def rec(prefix, left, dims):
            if dims == 1:
                layer.append(tuple(prefix + [left]))
                return
            for a in range(left, -1, -1):          # descending first component
                rec(prefix + [a], left - a, dims - 1)

        rec([], deg, D)
        out.extend(layer)
    return tuple(out)


def num_terms(D: int, p: int) -> int:
    """C(D+p-1, D): the O(D^p) coefficient count (Section 2)."""
    return math.comb(D + p - 1, D)


def mfact(alpha) -> float:
    """alpha! = prod alpha_d! (footnote 1)."""
    return float(np.prod([math.factorial(a) for a in alpha]))


def mpow(x: np.ndarray, alpha) -> np.ndarray:
    """x^alpha = prod_d x_d^alpha_d for x of shape (..., D)."""
    out = np.ones(x.shape[:-1])
    for d, a in enumerate(alpha):
        if a:
            out = out * x[..., d] ** a
    return out


# --------------------------------------------------------------------------
# Hermite functions (footnote 2)
# --------------------------------------------------------------------------
def hermite_polys(t: np.ndarray, nmax: int) -> np.ndarray:
    """H_0..H_nmax (physicists') at t, by H_{n+1} = 2t H_n - 2n H_{n-1}.
    Returns shape (nmax+1,) + t.shape."""
    t = np.asarray(t, dtype=np.float64)
    H = np.empty((nmax + 1,) + t.shape)
    H[0] = 1.0
    if nmax >= 1:
        H[1] = 2.0 * t
    for n in range(1, nmax):
        H[n + 1] = 2.0 * t * H[n] - 2.0 * n * H[n - 1]
    return H


def hermite_functions(t: np.ndarray, nmax: int) -> np.ndarray:
    """h_n(t) = e^{-t^2} H_n(t) for n = 0..nmax."""
    t = np.asarray(t, dtype=np.float64)
    return hermite_polys(t, nmax) * np.exp(-t * t)


def hermite_multi(t: np.ndarray, alpha) -> np.ndarray:
    """h_alpha(t) = prod_d h_{alpha_d}(t_d) for t of shape (..., D)."""
    out = np.ones(t.shape[:-1])
    for d, a in enumerate(alpha):
        out = out * hermite_functions(t[..., d], a)[a]
    return out


# --------------------------------------------------------------------------
# Far-field (Hermite) expansion about x_R (Section 1; Lemma 1's A_alpha)
# --------------------------------------------------------------------------
def hermite_coeffs(x_r: np.ndarray, w: np.ndarray, x_R: np.ndarray, h: float, p: int) -> np.ndarray:
    """A_alpha = sum_r w_r / alpha! ((x_r - x_R)/s)^alpha, |alpha| < p."""
    s = math.sqrt(2.0 * h * h)
    y = (np.asarray(x_r, np.float64) - x_R) / s
    return np.array([np.sum(w * mpow(y, a)) / mfact(a) for a in multi_indices(x_r.shape[1], p)])


def raw_moments(x_r: np.ndarray, w: np.ndarray, c: np.ndarray, p: int) -> np.ndarray:
    """Bandwidth-free moments M_alpha = sum_r w_r (x_r - c)^alpha / alpha!;
    A_alpha = M_alpha s^{-|alpha|}."""
    y = np.asarray(x_r, np.float64) - c
    return np.array([np.sum(w * mpow(y, a)) / mfact(a) for a in multi_indices(x_r.shape[1], p)])


def moments_to_hermite(Mraw: np.ndarray, D: int, p: int, h: float) -> np.ndarray:
    s = math.sqrt(2.0 * h * h)
    return np.array([Mraw[i] * s ** (-sum(a)) for i, a in enumerate(multi_indices(D, p))])


def eval_hermite(A: np.ndarray, x_R: np.ndarray, h: float, x_q: np.ndarray, p: int) -> np.ndarray:
    """EVALM / DH: sum_{|alpha|<p} A_alpha h_alpha((x_q - x_R)/s) per query."""
    s = math.sqrt(2.0 * h * h)
    t = (np.asarray(x_q, np.float64) - x_R) / s
    D = t.shape[1]
    return sum(A[i] * hermite_multi(t, a) for i, a in enumerate(multi_indices(D, p)))


# --------------------------------------------------------------------------
# Local (Taylor) expansion about x_Q (Section 1, second form; Lemma 5)
# --------------------------------------------------------------------------
def local_coeffs_direct(x_r: np.ndarray, w: np.ndarray, x_Q: np.ndarray, h: float, p: int) -> np.ndarray:
    """DIRECTL / DL: B_beta = 1/beta! sum_r w_r h_beta((x_r - x_Q)/s)."""
    s = math.sqrt(2.0 * h * h)
    v = (np.asarray(x_r, np.float64) - x_Q) / s
    return np.array([np.sum(w * hermite_multi(v, b)) / mfact(b)
                     for b in multi_indices(x_r.shape[1], p)])


def eval_local(B: np.ndarray, x_Q: np.ndarray, h: float, x_q: np.ndarray, p: int) -> np.ndarray:
    """EVALL: sum_{|beta|<p} B_beta ((x_q - x_Q)/s)^beta per query."""
    s = math.sqrt(2.0 * h * h)
    u = (np.asarray(x_q, np.float64) - x_Q) / s
    D = u.shape[1]
    return sum(B[i] * mpow(u, b) for i, b in enumerate(multi_indices(D, p)))


# --------------------------------------------------------------------------
# Translation operators (Section 3)
# --------------------------------------------------------------------------
def h2l(A: np.ndarray, x_R: np.ndarray, x_Q: np.ndarray, h: float, p_in: int, p_out: int) -> np.ndarray:
    """Lemma 1: B_beta = (-1)^{|beta|}/beta! sum_{|alpha|<p_in} A_alpha
    h_{alpha+beta}((x_Q - x_R)/s), for |beta| < p_out."""
    s = math.sqrt(2.0 * h * h)
    tau = ((np.asarray(x_Q, np.float64) - x_R) / s)[None, :]
    D = tau.shape[1]
    al = multi_indices(D, p_in)
    out = []
    for b in multi_indices(D, p_out):
        acc = 0.0
        for i, a in enumerate(al):
            ab = tuple(x + y for x, y in zip(a, b))
            acc += A[i] * hermite_multi(tau, ab)[0]
        out.append((-1.0) ** sum(b) / mfact(b) * acc)
    return np.array(out)


def h2h(A_child: np.ndarray, x_Rc: np.ndarray, x_R: np.ndarray, h: float, p: int) -> np.ndarray:
    """Lemma 2: A_gamma = sum_{alpha <= gamma} A'_alpha
    ((x_R' - x_R)/s)^{gamma-alpha} / (gamma-alpha)!."""
    s = math.sqrt(2.0 * h * h)
    delta = (np.asarray(x_Rc, np.float64) - x_R) / s
    D = delta.shape[0]
    al = multi_indices(D, p)
    out = []
    for g in al:
        acc = 0.0
        for i, a in enumerate(al):
            if all(x <= y for x, y in zip(a, g)):
                diff = tuple(y - x for x, y in zip(a, g))
                acc += A_child[i] * mpow(delta[None, :], diff)[0] / mfact(diff)
        out.append(acc)
    return np.array(out)


def l2l(B_parent: np.ndarray, x_Qp: np.ndarray, x_Q: np.ndarray, h: float, p: int) -> np.ndarray:
    """Lemma 3: B_alpha(child) = sum_{beta >= alpha} beta!/(alpha!(beta-alpha)!)
    B_beta ((x_Q - x_Q')/s)^{beta-alpha}."""
    s = math.sqrt(2.0 * h * h)
    delta = (np.asarray(x_Q, np.float64) - x_Qp) / s
    D = delta.shape[0]
    al = multi_indices(D, p)
    out = []
    for a in al:
        acc = 0.0
        for i, b in enumerate(al):
            if all(x <= y for x, y in zip(a, b)):
                diff = tuple(y - x for x, y in zip(a, b))
                acc += mfact(b) / (mfact(a) * mfact(diff)) * B_parent[i] * mpow(delta[None, :], diff)[0]
        out.append(acc)
    return np.array(out)


# --------------------------------------------------------------------------
# Truncation and finite-difference error bounds (Sections 4-5)
# --------------------------------------------------------------------------
def balanced_factor(D: int, p: int) -> float:
    """C(D+p-1, D-1) / sqrt((floor(p/D)!)^{D-p'} (ceil(p/D)!)^{p'}), p' = p mod D
    (the common factor of Lemmas 4-6)."""
    pp = p % D
    lo = math.factorial(p // D)
    hi = math.factorial(-(-p // D))
    return math.comb(D + p - 1, D - 1) / math.sqrt(float(lo ** (D - pp) * hi ** pp))


def bound_dh(p: int, D: int, W_R: float, dmin: float, h: float, r_R: float) -> float:
    """Lemma 4: E_DH(p); r_R = max_r ||x_r - x_R||_inf / h."""
    return W_R * math.exp(-dmin * dmin / (4 * h * h)) * balanced_factor(D, p) * r_R ** p


def bound_dl(p: int, D: int, W_R: float, dmin: float, h: float, r_Q: float) -> float:
    """Lemma 5: E_DL(p); r_Q = max_q ||x_q - x_Q||_inf / h."""
    return W_R * math.exp(-dmin * dmin / (4 * h * h)) * balanced_factor(D, p) * r_Q ** p


def bound_h2l(p: int, D: int, W_R: float, dmin: float, h: float, r_Q: float, r_R: float) -> float:
    """Lemma 6: E_H2L(p) = W_R e^{-dmin^2/4h^2} F(p) (r_Q^p + (sqrt2 r_R)^p
    C(D+p-1, D) (sqrt2 r_Q)^{I(sqrt2 r_Q)}), I(x) = 0 if x <= 1 else p-1."""
    x = math.sqrt(2.0) * r_Q
    expo = 0 if x <= 1.0 else p - 1
    tail = r_Q ** p + (math.sqrt(2.0) * r_R) ** p * math.comb(D + p - 1, D) * x ** expo
    return W_R * math.exp(-dmin * dmin / (4 * h * h)) * balanced_factor(D, p) * tail


def fd_estimate(W_R: float, dmin: float, dmax: float, h: float):
    """Section 5: G~_R = W_R (K(dmax) + K(dmin))/2 with error bound
    E_FD = W_R (K(dmin) - K(dmax))/2."""
    kmin = math.exp(-dmin * dmin / (2 * h * h))
    kmax = math.exp(-dmax * dmax / (2 * h * h))
    return W_R * (kmax + kmin) / 2, W_R * (kmin - kmax) / 2


def box_distances(lo_a, hi_a, lo_b, hi_b):
    """delta_min, delta_max between two axis-aligned boxes (Section 5)."""
    lo_a, hi_a, lo_b, hi_b = (np.asarray(v, np.float64) for v in (lo_a, hi_a, lo_b, hi_b))
    gap = np.maximum(0.0, np.maximum(lo_b - hi_a, lo_a - hi_b))
    far = np.maximum(hi_a - lo_b, hi_b - lo_a)
    return math.sqrt(float(np.sum(gap * gap))), math.sqrt(float(np.sum(far * far)))
