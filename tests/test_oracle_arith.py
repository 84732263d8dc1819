"""Pins of the oracle's ~212-bit arithmetic against exact rational arithmetic."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

REL = Fraction(1, 2 ** 200)


def rand_qd(rng, scale_exp=0):
    """A normalised 4-component value with random leading exponent."""
    hi = rng.uniform(0.5, 2.0) * 2.0 ** rng.randint(-20, 20) * rng.choice([-1, 1])
    terms = [hi]
    for _ in range(3):
        terms.append(terms[-1] * rng.uniform(-1, 1) * 2.0 ** -53)
    return oracle.qd_normalize(terms)


def test_normalize_is_exact_and_nonoverlapping():
    rng = random.Random(1)
    for _ in range(200):
        n = rng.randint(1, 24)
        t = [rng.uniform(-1, 1) * 2.0 ** rng.randint(-150, 10) for _ in range(n)]
        q = oracle.qd_normalize(t)
        exact = sum((Fraction(x) for x in t), Fraction(0))
        got = q.to_fraction()
        if exact == 0:
            assert got == 0
            continue
        assert abs(got - exact) <= abs(exact) * REL
        c = [x for x in q.c if x != 0.0]
        for a, b in zip(c, c[1:]):
            assert abs(b) <= math.ulp(a) / 2 * (1 + 1e-15)


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_binary_ops_exact_to_212_bits(op):
    rng = random.Random(hash(op) & 0xFFFF)
    for _ in range(300):
        a, b = rand_qd(rng), rand_qd(rng)
        fa, fb = a.to_fraction(), b.to_fraction()
        exact = {"add": fa + fb, "sub": fa - fb, "mul": fa * fb, "div": fa / fb}[op]
        got = oracle.qd_op(op, a.c, b.c).to_fraction()
        assert abs(got - exact) <= abs(exact) * REL * 16, op


def test_cancellation_in_add_is_exact():
    # a - a' for nearly equal a, a' keeps every bit of the difference.
    a = oracle.qd_normalize([1.0, 2.0 ** -60, 2.0 ** -130, 2.0 ** -190])
    b = oracle.qd_normalize([1.0, 2.0 ** -60, 2.0 ** -130, 0.0])
    d = oracle.qd_op("sub", a.c, b.c)
    assert d.to_fraction() == Fraction(2) ** -190


def test_rsqrt():
    rng = random.Random(7)
    for _ in range(200):
        a = rand_qd(rng)
        a = oracle.qd_normalize([abs(a.c[0])] + [x if a.c[0] > 0 else -x for x in a.c[1:]])
        x = oracle.qd_op("rsqrt", a.c).to_fraction()
        # x^2 a = 1 to within 2^-205
        assert abs(x * x * a.to_fraction() - 1) <= REL * 32


def test_det_matches_exact_rational():
    rng = np.random.default_rng(3)
    for d in (1, 2, 3, 5):
        re = rng.integers(-9, 10, size=(d, d)).astype(float)
        im = rng.integers(-9, 10, size=(d, d)).astype(float)
        A = re + 1j * im
        # exact complex determinant by the Leibniz formula over permutations
        from itertools import permutations
        tot_re, tot_im = Fraction(0), Fraction(0)
        for perm in permutations(range(d)):
            sgn = 1
            p = list(perm)
            for i in range(d):
                for j in range(i + 1, d):
                    if p[i] > p[j]:
                        sgn = -sgn
            pr, pi = Fraction(1), Fraction(0)
            for i in range(d):
                er, ei = Fraction(re[i, p[i]]), Fraction(im[i, p[i]])
                pr, pi = pr * er - pi * ei, pr * ei + pi * er
            tot_re += sgn * pr
            tot_im += sgn * pi
        gr, gi = oracle.det_qd(A)
        assert abs(gr.to_fraction() - tot_re) <= REL * (1 + abs(tot_re)) * 64
        assert abs(gi.to_fraction() - tot_im) <= REL * (1 + abs(tot_im)) * 64
