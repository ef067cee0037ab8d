"""Pins for the oracle's Alpert rule (Sec. 3.1, Sec. 4.1) against closed forms."""
import math
from decimal import Decimal

import numpy as np
import pytest

from oracle import alpert

# Textbook constants: Apery's constant zeta(3) and Glaisher-Kinkelin A.
ZETA3 = 1.2020569031595942854
GLAISHER = 1.2824271291006226369


def test_zeta_at_negative_integers_match_textbook_values():
    assert alpert.zeta_neg(0) == alpert.Fraction(-1, 2)
    assert alpert.zeta_neg(1) == alpert.Fraction(-1, 12)
    assert alpert.zeta_neg(2) == 0
    assert alpert.zeta_neg(3) == alpert.Fraction(1, 120)
    assert alpert.zeta_neg(5) == alpert.Fraction(-1, 252)


def test_zeta_prime_closed_forms():
    assert abs(float(alpert.zeta_prime_neg(0)) + 0.5 * math.log(2 * math.pi)) < 1e-15
    assert abs(float(alpert.zeta_prime_neg(1)) - (1.0 / 12.0 - math.log(GLAISHER))) < 1e-15
    assert abs(float(alpert.zeta_prime_neg(2)) + ZETA3 / (4 * math.pi ** 2)) < 1e-15


@pytest.mark.parametrize("order", [4, 8])
def test_rule_is_positive_and_inside_window(order):
    v, w, a = alpert.alpert_rule(order)
    assert len(v) == order - 1
    assert np.all(w > 0) and np.all(v > 0) and np.all(v < a)
    assert np.all(np.diff(v) > 0)
    # weight sum reproduces the dropped trapezoid weights: a - 1/2
    assert abs(np.sum(w) - (a - 0.5)) < 1e-14


def _log2sin(s):
    return np.log(np.abs(2.0 * np.sin(0.5 * s)))


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_fourier_cosine_integrals_of_log_kernel(n):
    # int_0^{2 pi} log|2 sin(t/2)| cos(n t) dt = -pi/n   (classical)
    for order, N, tol in ((4, 128, 2e-6 * n ** 4), (8, 64, 1e-9 * n ** 8)):
        I = alpert.corrected_periodic_integral(None, lambda s: _log2sin(s) * np.cos(n * s), N, order)
        assert abs(I + math.pi / n) < tol, (order, N, I + math.pi / n)


def test_constant_density_integral_is_zero():
    I = alpert.corrected_periodic_integral(None, _log2sin, 64, 4)
    assert abs(I) < 1e-7


def test_order_four_convergence_rate():
    f = lambda s: _log2sin(s) * np.exp(np.cos(s)) * 0 + _log2sin(s) * np.cos(2 * s)
    errs = [abs(alpert.corrected_periodic_integral(None, f, N, 4) + math.pi / 2) for N in (32, 64, 128)]
    rate1 = math.log2(errs[0] / errs[1])
    rate2 = math.log2(errs[1] / errs[2])
    # O(h^4 log h) -> observed rate a little below 4
    assert rate1 > 3.0 and rate2 > 3.0, errs


def test_circle_mean_log_distance():
    # (1/2pi) int log|x(0) - x(t)| dt = log R on a circle of radius R
    R = 0.7
    f = lambda s: np.log(R * np.abs(2.0 * np.sin(0.5 * s)))
    I = alpert.corrected_periodic_integral(None, f, 96, 4)
    assert abs(I / (2 * math.pi) - math.log(R)) < 1e-7


def test_lagrange_stencil_reproduces_polynomials():
    for t in (0.3, -0.3, 1.7, -2.9):
        offs, wts = alpert.lagrange_stencil(t, 6)
        assert t >= offs[0] - 1e-12 and t <= offs[-1] + 1e-12
        for p in range(6):
            assert abs(np.sum(wts * offs.astype(float) ** p) - t ** p) < 1e-11
    o1, _ = alpert.lagrange_stencil(0.4, 6)
    o2, _ = alpert.lagrange_stencil(-0.4, 6)
    assert np.array_equal(np.sort(-o2), o1)
