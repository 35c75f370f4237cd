"""Pins for the FP64 series-algebra reference (Sections 2-4).

The multi-index order is pinned by the paper's own worked example; the
Hermite functions by the Rodrigues formula of footnote 2 (sympy) and their
generating function; the expansions by convergence to the exhaustive oracle
with every truncation error under the Lemma 4/5/6 bound; H2H and L2L by
exactness against direct recomputation; FD by bracketing the true
contribution.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import exhaustive as ex
from oracle import series as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_graded_lex_matches_section2_worked_example():
    assert list(S.multi_indices(2, 2)) == _read_golden("graded_lex_d2_p2.txt")


def test_section2_moments_are_the_three_printed_sums():
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 1, (40, 2))
    w = rng.uniform(0.5, 1.5, 40)
    c = np.array([0.4, 0.6])
    h = 0.3
    s = math.sqrt(2 * h * h)
    A = S.hermite_coeffs(x, w, c, h, 2)
    want = [w.sum(), (w * (x[:, 0] - c[0]) / s).sum(), (w * (x[:, 1] - c[1]) / s).sum()]
    assert np.allclose(A, want, rtol=1e-14)


@pytest.mark.parametrize("D", range(1, 9))
def test_multi_index_set_count_and_order(D):
    for p in range(1, 7 if D > 4 else 9):
        al = S.multi_indices(D, p)
        brute = [a for a in itertools.product(range(p), repeat=D) if sum(a) < p]
        assert sorted(al) == sorted(brute)
        assert len(al) == S.num_terms(D, p) == math.comb(D + p - 1, D)
        # degree ascending; lexicographically descending within a degree
        keys = [(sum(a), tuple(-v for v in a)) for a in al]
        assert keys == sorted(keys)


def test_hermite_functions_match_rodrigues_formula():
    sympy = pytest.importorskip("sympy")
    t = sympy.symbols("t")
    g = sympy.exp(-t ** 2)
    pts = [-2.3, -0.7, 0.0, 0.4, 1.9, 3.1]
    vals = S.hermite_functions(np.array(pts), 12)
    deriv = g
    for n in range(13):
        hn = (-1) ** n * deriv           # h_n(t) = e^{-t^2} H_n(t) = (-1)^n D^n e^{-t^2}
        for i, tv in enumerate(pts):
            want = float(hn.subs(t, tv).evalf(30))
            assert vals[n, i] == pytest.approx(want, rel=1e-12, abs=1e-13)
        deriv = sympy.diff(deriv, t)


def test_hermite_generating_function():
    """sum_n h_n(t) s^n / n! = exp(-(t - s)^2)."""
    t = np.linspace(-3, 3, 13)
    for s in (-0.4, 0.1, 0.5):
        H = S.hermite_functions(t, 40)
        acc = sum(H[n] * s ** n / math.factorial(n) for n in range(41))
        assert np.allclose(acc, np.exp(-(t - s) ** 2), rtol=1e-12, atol=1e-14)


def test_cramer_inequality_with_constant_one():
    """|h_n(t)| <= 2^{n/2} sqrt(n!) e^{-t^2/2}: the inequality Lemmas 4-6 use."""
    t = np.linspace(-14, 14, 56001)
    H = S.hermite_functions(t, 18)
    for n in range(19):
        lhs = np.abs(H[n]) * np.exp(t * t / 2)
        assert lhs.max() <= 2 ** (n / 2) * math.sqrt(math.factorial(n)) * (1 + 1e-12), n


def _node(rng, n, D, center, half):
    x = center + rng.uniform(-half, half, (n, D))
    lo, hi = x.min(0), x.max(0)
    return x, lo, hi, (lo + hi) / 2


@pytest.mark.parametrize("D", [1, 2, 3, 5])
def test_far_field_converges_under_lemma4_bound(D):
    rng = np.random.default_rng(20 + D)
    h = 0.1
    xr, lor, hir, cR = _node(rng, 30, D, np.full(D, 0.3), 0.04)
    wr = rng.uniform(0.5, 1.5, 30)
    xq, loq, hiq, cQ = _node(rng, 25, D, np.full(D, 0.3 + 0.25 / math.sqrt(D)), 0.05)
    exact = ex.gauss_sum(xq, xr, wr, [h])[:, 0]
    dmin, _ = S.box_distances(loq, hiq, lor, hir)
    rR = float(np.max(np.abs(xr - cR))) / h
    errs = []
    for p in range(1, 9 if D < 5 else 7):
        A = S.hermite_coeffs(xr, wr, cR, h, p)
        err = np.max(np.abs(S.eval_hermite(A, cR, h, xq, p) - exact))
        assert err <= S.bound_dh(p, D, wr.sum(), dmin, h, rR) * (1 + 1e-9) + 1e-15
        errs.append(err)
    # converges towards the exhaustive sum as p grows
    assert errs[-1] < errs[0] / 50 and errs[-1] < 1e-2 * exact.min()


@pytest.mark.parametrize("D", [1, 2, 3, 5])
def test_direct_local_converges_under_lemma5_bound(D):
    rng = np.random.default_rng(30 + D)
    h = 0.1
    xr, lor, hir, cR = _node(rng, 20, D, np.full(D, 0.5), 0.05)
    wr = rng.uniform(0.5, 1.5, 20)
    xq, loq, hiq, cQ = _node(rng, 40, D, np.full(D, 0.5 - 0.2 / math.sqrt(D)), 0.04)
    exact = ex.gauss_sum(xq, xr, wr, [h])[:, 0]
    dmin, _ = S.box_distances(loq, hiq, lor, hir)
    rQ = float(np.max(np.abs(xq - cQ))) / h
    errs = []
    for p in range(1, 9 if D < 5 else 7):
        B = S.local_coeffs_direct(xr, wr, cQ, h, p)
        err = np.max(np.abs(S.eval_local(B, cQ, h, xq, p) - exact))
        assert err <= S.bound_dl(p, D, wr.sum(), dmin, h, rQ) * (1 + 1e-9) + 1e-15
        errs.append(err)
    assert errs[-1] < errs[0] / 50 and errs[-1] < 1e-2 * exact.min()


@pytest.mark.parametrize("D", [1, 2, 3])
def test_h2l_converges_under_lemma6_bound(D):
    rng = np.random.default_rng(40 + D)
    h = 0.1
    xr, lor, hir, cR = _node(rng, 25, D, np.full(D, 0.2), 0.03)
    wr = rng.uniform(0.5, 1.5, 25)
    xq, loq, hiq, cQ = _node(rng, 25, D, np.full(D, 0.2 + 0.3 / math.sqrt(D)), 0.03)
    exact = ex.gauss_sum(xq, xr, wr, [h])[:, 0]
    dmin, _ = S.box_distances(loq, hiq, lor, hir)
    rQ = float(np.max(np.abs(xq - cQ))) / h
    rR = float(np.max(np.abs(xr - cR))) / h
    errs = []
    for p in range(1, 8 if D < 3 else 6):
        A = S.hermite_coeffs(xr, wr, cR, h, p)
        B = S.h2l(A, cR, cQ, h, p, p)
        err = np.max(np.abs(S.eval_local(B, cQ, h, xq, p) - exact))
        assert err <= S.bound_h2l(p, D, wr.sum(), dmin, h, rQ, rR) * (1 + 1e-9) + 1e-15
        errs.append(err)
    assert errs[-1] < errs[0] / 50 and errs[-1] < 1e-2 * exact.min()


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_h2h_is_exact(D):
    """Moments of the union about the parent centre equal the H2H-shifted
    moments of the two children, term by term (Lemma 2 is exact)."""
    rng = np.random.default_rng(50 + D)
    h, p = 0.07, 6
    x1, *_ , c1 = _node(rng, 15, D, np.full(D, 0.3), 0.05)
    x2, *_ , c2 = _node(rng, 12, D, np.full(D, 0.45), 0.05)
    w1, w2 = rng.uniform(0.5, 1.5, 15), rng.uniform(0.5, 1.5, 12)
    c = (c1 + c2) / 2
    direct = S.hermite_coeffs(np.vstack([x1, x2]), np.concatenate([w1, w2]), c, h, p)
    shifted = (S.h2h(S.hermite_coeffs(x1, w1, c1, h, p), c1, c, h, p)
               + S.h2h(S.hermite_coeffs(x2, w2, c2, h, p), c2, c, h, p))
    assert np.allclose(shifted, direct, rtol=1e-11, atol=1e-13 * np.abs(direct).max())


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_l2l_is_exact(D):
    """A shifted local expansion is the same polynomial (Lemma 3 is exact)."""
    rng = np.random.default_rng(60 + D)
    h, p = 0.1, 6
    B = rng.standard_normal(S.num_terms(D, p))
    cp = rng.uniform(0, 1, D)
    cc = cp + rng.uniform(-0.05, 0.05, D)
    xq = cc + rng.uniform(-0.03, 0.03, (20, D))
    a = S.eval_local(B, cp, h, xq, p)
    b = S.eval_local(S.l2l(B, cp, cc, h, p), cc, h, xq, p)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(a).max())


def test_order_one_special_cases():
    rng = np.random.default_rng(70)
    D, h = 3, 0.2
    c = np.array([0.5, 0.5, 0.5])
    xr = np.tile(c, (10, 1))                       # every reference at the centre
    wr = rng.uniform(0.5, 1.5, 10)
    xq = rng.uniform(0, 1, (8, D))
    exact = ex.gauss_sum(xq, xr, wr, [h])[:, 0]
    A = S.hermite_coeffs(xr, wr, c, h, 1)
    assert np.allclose(S.eval_hermite(A, c, h, xq, 1), exact, rtol=1e-13)   # DH p=1 exact
    B = S.local_coeffs_direct(rng.uniform(0, 1, (6, D)), np.ones(6), c, h, 4)
    assert S.eval_local(B, c, h, c[None, :], 4)[0] == pytest.approx(B[0], rel=1e-15)  # at x_Q


def test_balanced_factor_small_cases():
    # p = 1: C(D, D-1) / sqrt(1) = D ; D = 1: C(p, 0)/sqrt(p!) = 1/sqrt(p!)
    for D in range(2, 9):
        assert S.balanced_factor(D, 1) == D
    for p in range(1, 8):
        assert S.balanced_factor(1, p) == pytest.approx(1 / math.sqrt(math.factorial(p)))
    # D = 2, p = 3: p' = 1, floor = 1, ceil = 2 -> C(4,1)/sqrt(1 * 2) = 4/sqrt 2
    assert S.balanced_factor(2, 3) == pytest.approx(4 / math.sqrt(2))


def test_lemma_bounds_hand_values():
    """Lemmas 4-6 evaluated by hand for one node pair, so that a bound that
    is too loose (a dropped sqrt 2, a wrong binomial, the I() exponent on the
    wrong term) fails, not only one that is too tight.  D = 2, p = 3:
    p' = 1, floor(p/D)! = 1, ceil(p/D)! = 2, C(D+p-1, D-1) = C(4, 1) = 4, so
    the common factor is 4 / sqrt(1 * 2) = 2 sqrt 2; C(D+p-1, D) = C(4, 2) = 6.
    W_R = 2.5, delta_min = 0.6, h = 0.5: e^{-delta^2 / 4h^2} = e^{-0.36}.
    Lemma 6's I() multiplies the term that carries C(D+p-1, D): it counts the
    Taylor terms |beta| < p of the converted expansion, each at most
    (sqrt 2 r_Q)^{|beta|} (the E_1 part of the proof)."""
    e = math.exp(-0.36)
    r2 = math.sqrt(2.0)
    # E_DH, r_R = 0.4: 2.5 * 2 sqrt2 * 0.064 = 0.32 sqrt2
    assert S.bound_dh(3, 2, 2.5, 0.6, 0.5, 0.4) == pytest.approx(0.32 * r2 * e, rel=1e-14)
    # E_DL, r_Q = 0.3: 2.5 * 2 sqrt2 * 0.027 = 0.135 sqrt2
    assert S.bound_dl(3, 2, 2.5, 0.6, 0.5, 0.3) == pytest.approx(0.135 * r2 * e, rel=1e-14)
    # E_H2L, r_Q = 0.3 (sqrt2 r_Q <= 1: I = 0), r_R = 0.4:
    #   5 sqrt2 (0.027 + (0.4 sqrt2)^3 * 6) = 5 sqrt2 (0.027 + 0.768 sqrt2) = 0.135 sqrt2 + 7.68
    assert S.bound_h2l(3, 2, 2.5, 0.6, 0.5, 0.3, 0.4) == pytest.approx((0.135 * r2 + 7.68) * e, rel=1e-14)
    # E_H2L, r_Q = 0.8 (sqrt2 r_Q > 1: I = p - 1 = 2, (0.8 sqrt2)^2 = 1.28):
    #   5 sqrt2 (0.512 + 0.768 sqrt2 * 1.28) = 2.56 sqrt2 + 9.8304
    assert S.bound_h2l(3, 2, 2.5, 0.6, 0.5, 0.8, 0.4) == pytest.approx((2.56 * r2 + 9.8304) * e, rel=1e-14)
    # D = 3, p = 4: p' = 1, factor C(6, 2) / sqrt(1 * 1 * 2) = 15 / sqrt2; at delta_min = 0
    assert S.bound_dh(4, 3, 1.0, 0.0, 1.0, 0.5) == pytest.approx(15 / r2 * 0.0625, rel=1e-14)
    # D = 5, p = 7: p' = 2, floor = 1, ceil = 2 -> sqrt(1^3 * 2^2) = 2, C(11, 4) = 330 -> 165
    assert S.balanced_factor(5, 7) == pytest.approx(165.0, rel=1e-15)


def test_fd_estimate_brackets_the_true_contribution():
    rng = np.random.default_rng(80)
    for trial in range(20):
        D = int(rng.integers(1, 6))
        h = float(rng.uniform(0.05, 0.5))
        xr, lor, hir, _ = _node(rng, 20, D, rng.uniform(0, 1, D), 0.05)
        xq, loq, hiq, _ = _node(rng, 10, D, rng.uniform(0, 1, D), 0.05)
        wr = rng.uniform(0.5, 1.5, 20)
        dmin, dmax = S.box_distances(loq, hiq, lor, hir)
        est, err = S.fd_estimate(wr.sum(), dmin, dmax, h)
        exact = ex.gauss_sum(xq, xr, wr, [h])[:, 0]
        assert np.all(np.abs(exact - est) <= err * (1 + 1e-12) + 1e-15)


def test_box_distances_bound_every_point_pair():
    rng = np.random.default_rng(90)
    for trial in range(20):
        D = int(rng.integers(1, 5))
        xa = rng.uniform(0, 1, (8, D)) * rng.uniform(0.1, 0.5) + rng.uniform(0, 1, D)
        xb = rng.uniform(0, 1, (9, D)) * rng.uniform(0.1, 0.5) + rng.uniform(0, 1, D)
        dmin, dmax = S.box_distances(xa.min(0), xa.max(0), xb.min(0), xb.max(0))
        d = np.sqrt(((xa[:, None, :] - xb[None, :, :]) ** 2).sum(-1))
        assert d.min() >= dmin - 1e-12 and d.max() <= dmax + 1e-12
        # the box corners attain delta_max
        ca = np.array(list(itertools.product(*zip(xa.min(0), xa.max(0)))))
        cb = np.array(list(itertools.product(*zip(xb.min(0), xb.max(0)))))
        dc = np.sqrt(((ca[:, None, :] - cb[None, :, :]) ** 2).sum(-1))
        assert dc.max() == pytest.approx(dmax, rel=1e-12)
