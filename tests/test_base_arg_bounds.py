"""CPU pin of the direct base-case kernel's exponent-argument error bound.

The direct kernel forms c ||q - r||^2 + l as fma(d2, c, l) with d2 an FMA
chain of the rounded coordinate differences; its charge per term is
(D+5) u |arg| (the differences 2, the chain D, c 1, the FMA 1, the rounding
of l 1).  This test replays that exact sequence of FP32 operations in exact
rational arithmetic (every operation rounded once to FP32,
round-to-nearest-even) on random leaf pairs and checks the bound against the
exact argument.
"""

from fractions import Fraction as Fr
import math

import numpy as np
import pytest


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
