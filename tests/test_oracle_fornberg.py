"""Pins for oracle.fornberg: Fornberg coefficients, modified wave numbers, centering symbol.

Each check is against something other than the oracle's own formula: textbook
finite-difference / Lagrange weights, polynomial exactness by brute force,
trigonometric closed forms, or the infinite-order limit.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fornberg


def test_alpha_staggered_textbook_values():
    # m = 1: the two-point midpoint average / difference.
    assert fornberg.alpha_staggered(1) == [Fraction(1)]
    # m = 2: fourth-order staggered derivative (27 (f_{1/2} - f_{-1/2}) - (f_{3/2} - f_{-3/2})) / 24;
    # as interpolation weights alpha/2 = {9/16, -1/16}, the 4-point midpoint Lagrange rule.
    assert fornberg.alpha_staggered(2) == [Fraction(9, 8), Fraction(-1, 8)]
    assert [a / 2 for a in fornberg.alpha_staggered(2)] == [Fraction(9, 16), Fraction(-1, 16)]
    assert fornberg.alpha_staggered(4) == [Fraction(1225, 1024), Fraction(-245, 1024),
                                           Fraction(49, 1024), Fraction(-5, 1024)]


def test_alpha_centered_textbook_values():
    # m = 1: (f_1 - f_-1) / 2; m = 2: (8 (f_1 - f_-1) - (f_2 - f_-2)) / 12.
    assert fornberg.alpha_centered(1) == [Fraction(1)]
    assert fornberg.alpha_centered(2) == [Fraction(4, 3), Fraction(-1, 3)]


def _lagrange_midpoint_weights(m):
    """Brute force: weights of the degree-(2m-1) Lagrange interpolant through the nodes
    +-1/2, +-3/2, ... evaluated at 0 (weights for the nodes n - 1/2, n = 1..m)."""
    nodes = [Fraction(2 * n - 1, 2) for n in range(1, m + 1)]
    nodes = nodes + [-x for x in nodes]
    w = []
    for xi in nodes[:m]:
        p = Fraction(1)
        for xj in nodes:
            if xj != xi:
                p *= (0 - xj) / (xi - xj)
        w.append(p)
    return w


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6, 8])
def test_centering_weights_are_lagrange_interpolation(m):
    # alpha^s/2 must be the symmetric Lagrange weights (interpolation exact to degree 2m-1).
    assert [a / 2 for a in fornberg.alpha_staggered(m)] == _lagrange_midpoint_weights(m)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_staggered_moment_property(m):
    # Eq. eq_Fornberg_property holds for k = 0 .. m-1 (exact rationals).  The paper states it
    # up to k = m; the k = m moment is not zero, so centering is O(dx^{2m}) (reading recorded).
    a = fornberg.alpha_staggered(m)
    for k in range(m):
        s = sum(a[n - 1] * Fraction(2 * n - 1, 2) ** (2 * k) for n in range(1, m + 1))
        assert s == (1 if k == 0 else 0)
    s = sum(a[n - 1] * Fraction(2 * n - 1, 2) ** (2 * m) for n in range(1, m + 1))
    assert s != 0
    if m == 2:
        assert s == Fraction(-9, 16)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_staggered_derivative_exact_on_polynomials(m):
    # Eq. staggered_finite_difference differentiates polynomials of degree <= 2m exactly.
    a = fornberg.alpha_staggered(m)
    for deg in range(0, 2 * m + 1):
        f = lambda x: x ** deg
        d = sum(a[n - 1] * (f(Fraction(2 * n - 1, 2)) - f(-Fraction(2 * n - 1, 2))) / (2 * n - 1)
                for n in range(1, m + 1))
        assert d == (1 if deg == 1 else 0)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_centered_derivative_exact_on_polynomials(m):
    a = fornberg.alpha_centered(m)
    for deg in range(0, 2 * m + 1):
        d = sum(a[n - 1] * (Fraction(n) ** deg - Fraction(-n) ** deg) / (2 * n) for n in range(1, m + 1))
        assert d == (1 if deg == 1 else 0)


def test_modified_wave_numbers_order2_closed_form():
    N, dx = 16, 0.3
    k = fornberg.wave_numbers(N, dx)
    ks = fornberg.k_staggered(N, dx, 2).astype(float)
    kc = fornberg.k_centered(N, dx, 2).astype(float)
    np.testing.assert_allclose(ks, 2 * np.sin(k * dx / 2) / dx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(kc, np.sin(k * dx) / dx, rtol=0, atol=1e-14)
    assert kc[N // 2] == 0.0              # exact zero at Nyquist


def test_modified_wave_numbers_converge_to_k():
    N, dx = 64, 1.0
    k = fornberg.wave_numbers(N, dx)
    inner = np.abs(k * dx) <= np.pi / 2
    for order, tol in [(16, 1e-3), (64, 1e-9)]:
        ks = fornberg.k_staggered(N, dx, order).astype(float)
        kc = fornberg.k_centered(N, dx, order).astype(float)
        assert np.max(np.abs(ks - k)[inner]) < tol
        assert np.max(np.abs(kc - k)[inner]) < 100 * tol
    np.testing.assert_allclose(fornberg.k_staggered(N, dx, 0).astype(float), k, rtol=1e-15, atol=0)


def test_zeta_special_values_and_limit():
    N = 32
    for order in (2, 4, 8, 16):
        z = fornberg.zeta(N, order).astype(float)
        assert z[0] == 1.0
        assert z[N // 2] == 0.0
        assert np.all(z <= 1.0 + 1e-15)
    # order 2: zeta = cos(k dx / 2) (the two-point average)
    k = fornberg.wave_numbers(N, 1.0)
    np.testing.assert_allclose(fornberg.zeta(N, 2).astype(float), np.cos(k / 2), atol=1e-15)
    # zeta -> 1 as the order grows, at k dx = pi/2
    q = N // 4
    vals = [float(fornberg.zeta(N, o)[q]) for o in (2, 4, 8, 16, 32)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    assert vals[3] > 0.998 and vals[-1] > 0.99999      # order 16 and order 32
