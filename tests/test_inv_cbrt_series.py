"""The correction the neo-Hookean law applies to a single-precision
J^{-1/3} (App. A, eq. neoHook: r = J^{-1/3} scales the isochoric and
volumetric terms), checked on the host with every FP64 operation rounded
exactly as the device does it (products, sums and fused multiply-adds taken
in exact rational arithmetic and rounded once): for estimates off by up to
four single-precision units in the last place, r (1 + h/3 + 2h^2/9) with
h = 1 - J r^3 lands within 1.5 double-precision units of the exact J^{-1/3}
(computed to 50 digits), and a correction that drops the h^2 term or uses
the wrong series coefficient does not."""
from __future__ import annotations

import decimal
from fractions import Fraction

import numpy as np


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _mul(a, b):
    return float(Fraction(a) * Fraction(b))


def _corrected(J, r, c2=2.0 / 9.0, c1=1.0 / 3.0):
    r3 = _mul(_mul(r, r), r)
    h = _fma(-J, r3, 1.0)
    t = _mul(h, _fma(h, c2, c1))
    return _fma(r, t, r)


def _exact(J):
    decimal.getcontext().prec = 50
    return decimal.Decimal(J) ** (decimal.Decimal(-1) / decimal.Decimal(3))


def _ulps(x, ref):
    return float(abs(decimal.Decimal(x) - ref) / decimal.Decimal(np.spacing(float(ref))))


def _estimates(J):
    r32 = np.float32(float(_exact(J)))
    for k in (-4, -1, 0, 1, 4):
        yield float(np.float32(r32 + np.float32(k) * np.spacing(r32)))


def test_series_correction_reaches_double_precision():
    rng = np.random.default_rng(1)
    Js = list(10.0 ** rng.uniform(-3.0, 3.0, 300)) + [1.0, 8.0, 0.125, 1.0 + 2.0 ** -40, 27.0]
    worst = 0.0
    for J in Js:
        ref = _exact(J)
        for r0 in _estimates(J):
            worst = max(worst, _ulps(_corrected(J, r0), ref))
    assert worst <= 1.5, worst


def test_series_correction_needs_both_terms():
    J = 3.7
    ref = _exact(J)
    r0 = next(iter(_estimates(J)))  # four units low
    assert _ulps(_corrected(J, r0), ref) <= 1.5
    assert _ulps(_corrected(J, r0, c2=0.0), ref) > 4.0        # first-order step only
    assert _ulps(_corrected(J, r0, c1=1.0 / 2.0), ref) > 1e6  # wrong leading coefficient
