"""The inverse square roots of the FP64 trees, checked one value at a time against exact values.

The FP64 kernels form every det(P)^(-1/2) without FP64 instructions (an FP32 seed and one exact
integer Newton step, accurate to about 0.51 units in the last place).  Two trees expose them:

* one mode, G = P (2 x 2): the tree's included sum is exactly d^(-1/2), with d the FP64
  determinant fma(p00, p11, -fl(p10^2));
* two modes, G = diag(P_a, I) with P_a = diag(x, 1): the pivot of mode a is factored as
  r0 = x^(-1/2), r1 = 1, and the included sum is exactly r0 - 1.

Each result is compared with the exact inverse square root (rational determinant, 60-digit
square root): |g - exact| <= 0.51 ulp(g).
"""
import decimal
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import paper_1810_00900_gb300 as gbs
from helpers import frac3

pytestmark = pytest.mark.gpu
decimal.getcontext().prec = 60


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def inv_sqrt_exact(q: Fraction) -> Fraction:
    d = decimal.Decimal(q.numerator) / decimal.Decimal(q.denominator)
    return Fraction(1 / d.sqrt())


def ulp(g: float) -> float:
    return math.ldexp(1.0, math.frexp(g)[1] - 53)


def check(g, exact, what):
    assert abs(Fraction(g) - exact) <= Fraction(0.51) * Fraction(ulp(g)), (what, g, float(exact))


def pivots(seed, count):
    rnd = random.Random(seed)
    out = [(1.0, 1.0, 0.0), (0.25, 1.0, 0.0), (4.0, 0.25, 0.5), (2.0, 2.0, 1.0), (1.0, 1.0, 0.999999)]
    for _ in range(count):
        a = math.ldexp(rnd.uniform(0.5, 2.0), rnd.randint(-40, 40))
        c = math.ldexp(rnd.uniform(0.5, 2.0), rnd.randint(-40, 40))
        rho = rnd.choice([rnd.uniform(-1, 1), rnd.uniform(-1, 1) * 1e-3, 1 - 10 ** rnd.uniform(-12, -1), 0.0])
        out.append((a, c, rho * math.sqrt(a * c)))
    return out


def test_leaf_determinant_inverse_square_root(ctx):
    for p00, p11, p10 in pivots(7, 200):
        G = np.array([[p00, p10], [p10, p11]])
        inc, exc, _, _ = gbs.subset_sum(ctx, G, "real", "fp64")
        g = frac3(inc)
        assert frac3(exc) == -1
        det = float(Fraction(p00) * Fraction(p11) - Fraction(p10 * p10))  # one rounding, as the FMA
        check(float(g), inv_sqrt_exact(Fraction(det)), (p00, p11, p10))
        assert g == Fraction(float(g))  # a single double


def test_pivot_inverse_square_root(ctx):
    rnd = random.Random(11)
    xs = [1.0, 0.25, 4.0, 2.0, 0.5, 3.999999999999999, 1.0000000000000002, 0.9999999999999999]
    xs += [math.ldexp(rnd.uniform(1.0, 2.0), rnd.randint(-300, 300)) for _ in range(200)]
    for x in xs:
        G = np.diag([x, 1.0, 1.0, 1.0])
        inc, _, _, _ = gbs.subset_sum(ctx, G, "real", "fp64")
        g = frac3(inc) + 1
        check(float(g), inv_sqrt_exact(Fraction(x)), x)


def test_not_positive_definite_pivots(ctx):
    for G in (np.array([[-1.0, 0.0], [0.0, 1.0]]), np.array([[1.0, 2.0], [2.0, 1.0]]),
              np.array([[-1.0, 0.0], [0.0, -1.0]])):
        with pytest.raises(gbs.GbsError):
            gbs.subset_sum(ctx, G, "real", "fp64")
