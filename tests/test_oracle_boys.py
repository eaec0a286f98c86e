"""Pins for the oracle's Boys function (paper Eq. boys_function).

F_m(x) = int_0^1 t^(2m) exp(-x t^2) dt is checked against 40-digit mpmath
quadrature of that definition, against its value at x = 0, against its
large-x asymptote, and against the downward recurrence identity.
"""
import math

import numpy as np
import pytest

import oracle


def test_boys_at_zero():
    F = oracle.boys(13, 0.0)
    for m in range(14):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


def test_boys_vs_mpmath_quadrature():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    xs = [1e-8, 1e-4, 0.01, 0.3, 1.0, 2.5, 7.0, 12.0, 19.9, 29.9, 30.0, 30.1, 45.0, 80.0, 200.0]
    worst = 0.0
    for x in xs:
        F = oracle.boys(13, x)
        for m in range(14):
            ref = mp.quad(lambda t: t ** (2 * m) * mp.e ** (-x * t * t), [0, mp.mpf(1) / 2, 1])
            rel = abs(F[m] - float(ref)) / float(ref)
            worst = max(worst, rel)
            assert rel < 4e-15, (x, m, F[m], float(ref))
    assert worst < 4e-15


def test_boys_asymptote():
    # F_m(x) -> (2m-1)!! / 2^(m+1) * sqrt(pi / x^(2m+1)) for x >> m (error ~ exp(-x))
    x = 300.0
    F = oracle.boys(13, x)
    for m in range(14):
        dfac = math.prod(range(2 * m - 1, 0, -2)) if m > 0 else 1
        ref = dfac / 2 ** (m + 1) * math.sqrt(math.pi / x ** (2 * m + 1))
        assert F[m] == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("x", [0.05, 1.7, 9.0, 24.0, 33.0, 60.0])
def test_boys_downward_identity(x):
    F = oracle.boys(13, x)
    for m in range(13):
        assert F[m] == pytest.approx((2 * x * F[m + 1] + math.exp(-x)) / (2 * m + 1), rel=2e-14)
