"""CPU pins of the base-case kernels' exponent-argument error bounds.

The direct kernel forms c ||q - r||^2 + l as fma(d2, c, l) with d2 an FMA
chain of the rounded coordinate differences; its charge per term is
(D+5) u |arg| (the differences 2, the chain D, c 1, the FMA 1, the rounding
of l 1).  The expanded-distance kernel forms the exponent argument c ||q - r||^2 + l as
c ((|v|^2 - 2 u.v) + |u|^2) + l with u = q - c_R, v = r - c_R about the
reference leaf's FP32 centre, in FP32 with fused multiply-adds.  This test
replays that exact sequence of FP32 operations in exact rational arithmetic
(every operation rounded once to FP32, round-to-nearest-even) on random and
adversarial leaf pairs and checks the first-order bound the library charges
(oracle.dualtree.xp_arg_bound plus the rounding of l) against the exact
argument.  A dropped term in the bound (the input roundings, the |u|^2
chain, the final FMA) or a wrong anchor radius fails it.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

from oracle import dualtree as T

U = 2.0 ** -24


def rnd32(x: Fr) -> Fr:
    """Round an exact rational to the nearest FP32 value (ties to even);
    normal range only."""
    if x == 0:
        return Fr(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    scale = Fr(2) ** (23 - e)
    m = a * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    return s * Fr(fl) / scale


def f32(x: float) -> Fr:
    return Fr(float(np.float32(x)))


def kernel_arg(q, r, c, cf, l):
    """The kernel's FP32 operations, each rounded once: v = fl(r - c),
    m = -2 v, s = |v|^2 by an FMA chain, u = fl(q - c), b = |u|^2 by an FMA
    chain, t = fma chain of u_d m_d onto s, t = fl(t + b), arg = fma(t, cf, l)."""
    D = len(q)
    v = [rnd32(r[d] - c[d]) for d in range(D)]
    m = [-2 * vd for vd in v]
    s = rnd32(v[0] * v[0])
    for d in range(1, D):
        s = rnd32(v[d] * v[d] + s)
    u = [rnd32(q[d] - c[d]) for d in range(D)]
    b = rnd32(u[0] * u[0])
    for d in range(1, D):
        b = rnd32(u[d] * u[d] + b)
    t = s
    for d in range(D):
        t = rnd32(u[d] * m[d] + t)
    t = rnd32(t + b)
    return rnd32(t * cf + l)


def direct_arg(q, r, cf, l):
    """The direct kernel's FP32 operations: df = fl(q - r), d2 = fl(df_0^2)
    then FMAs, arg = fma(d2, cf, l)."""
    D = len(q)
    df = [rnd32(q[d] - r[d]) for d in range(D)]
    d2 = rnd32(df[0] * df[0])
    for d in range(1, D):
        d2 = rnd32(df[d] * df[d] + d2)
    return rnd32(d2 * cf + l)


def _case(rng, D, h, rho_frac, d_frac, centre_scale):
    """A reference leaf of Euclidean radius about rho_frac * h around an FP32
    centre at |centre| ~ centre_scale, a reference point in it and a query at
    distance about d_frac * h from that point."""
    cen = rng.uniform(-1.0, 1.0, D) * centre_scale
    c = [f32(x) for x in cen]
    pts = []
    for _ in range(4):
        dirv = rng.standard_normal(D)
        dirv /= np.linalg.norm(dirv)
        pts.append(np.array([float(x) for x in c]) + dirv * rho_frac * h * rng.uniform(0.2, 1.0))
    pts = [[f32(x) for x in p] for p in pts]
    rho = max(math.sqrt(sum(float(p[d] - c[d]) ** 2 for d in range(D))) for p in pts) * (1 + 1e-12)
    r = pts[0]
    dirq = rng.standard_normal(D)
    dirq /= np.linalg.norm(dirq)
    q = [f32(float(r[d]) + dirq[d] * d_frac * h) for d in range(D)]
    return q, r, c, rho


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8])
def test_expanded_argument_within_bound(D):
    rng = np.random.default_rng(1206685700 + D)
    worst = 0.0
    for k in range(150):
        h = float(10.0 ** rng.uniform(-4, 0))
        rho_frac = float(10.0 ** rng.uniform(-2, 2))          # leaf radius from 0.01 h to 100 h
        d_frac = float(rng.choice([0.0, 1e-3, 0.3, 2.0, 9.42]) * rng.uniform(0.5, 1.0))
        centre_scale = float(10.0 ** rng.uniform(-1, 2))
        q, r, c, rho = _case(rng, D, h, rho_frac, d_frac, centre_scale)
        cexact = -1.4426950408889634 / (2.0 * h * h)
        cf = f32(cexact)
        w = float(rng.uniform(0.01, 1.0))
        lexact = math.log2(w)
        l = f32(lexact)
        got = kernel_arg(q, r, c, cf, l)
        d2 = sum((q[i] - r[i]) ** 2 for i in range(D))
        exact = Fr(cexact) * d2 + Fr(lexact)
        d = math.sqrt(float(d2))
        bound = T.xp_arg_bound(D, d, rho, cexact, float(exact)) + U * abs(lexact)
        err = abs(float(got - exact))
        assert err <= bound * (1 + 1e-9) + 1e-300, (D, h, rho_frac, d_frac, err, bound)
        worst = max(worst, err / bound if bound > 0 else 0.0)
    assert worst > 0.0


def test_guard_threshold_matches_bound():
    """The guard's coefficients dominate the bound's absolute part at
    d = 9.42 h: (4D+7) 9.42 x + (5D+2) x^2 >= (4D+4) 9.42 x + 5D x^2 for
    x = rho_R / h, and at d = 9.42 h the term is 2^-64: c d^2 >= 64."""
    for D in range(1, 9):
        for x in (0.01, 1.0, 20.0):
            assert (4 * D + 7) * 9.42 * x + (5 * D + 2) * x * x >= (4 * D + 4) * 9.42 * x + 5 * D * x * x
    assert 1.4426950408889634 / 2.0 * 9.42 ** 2 >= 64.0


def test_xp_charge_and_enabling():
    u = U
    assert T.xp_rho() == pytest.approx(math.log(2) * (128 * u + 2.0 ** -13), rel=1e-15)
    assert T.xp_enabled(3, True, 32, 64, 64)
    assert not T.xp_enabled(3, True, 32, 32, 64)      # one query per lane: scalar kernel
    assert not T.xp_enabled(3, False, 32, 64, 64)     # FP64 points
    assert not T.xp_enabled(9, True, 32, 64, 64)
    assert not T.xp_enabled(3, True, 33, 64, 64)
    assert not T.xp_enabled(3, True, 32, 64, 64, no_xp=True)
    base = T.fp32_rho(3, 1000, 1.0, 1000.0, -40, 64)
    assert T.fp32_rho(3, 1000, 1.0, 1000.0, -40, 64, xp=True) == pytest.approx(base + T.xp_rho(), rel=1e-15)


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8, 16])
def test_direct_argument_within_charge(D):
    """Per term, |arg~ - arg| <= (D+5) u |arg|: the relative argument error
    the FP32 charge takes over exponents down to 2^-64 (ln2 64 (D+5) u)."""
    rng = np.random.default_rng(1206685800 + D)
    for k in range(200):
        h = float(10.0 ** rng.uniform(-4, 0))
        q, r, c, rho = _case(rng, D, h, float(10.0 ** rng.uniform(-2, 1)),
                             float(rng.uniform(0.0, 9.42)), float(10.0 ** rng.uniform(-1, 2)))
        cexact = -1.4426950408889634 / (2.0 * h * h)
        lexact = math.log2(float(rng.uniform(0.01, 1.0)))
        got = direct_arg(q, r, f32(cexact), f32(lexact))
        exact = Fr(cexact) * sum((q[i] - r[i]) ** 2 for i in range(D)) + Fr(lexact)
        err = abs(float(got - exact))
        assert err <= (D + 5) * U * abs(float(exact)) * (1 + 1e-9), (D, err, float(exact))
