"""Fornberg coefficients, modified wave numbers and the centering symbol.

Test infrastructure only (see oracle/__init__.py).

* alpha_staggered(m): Eq. eq_Fornberg_staggered (Sec. 4.1; also Sec. 3).
* alpha_centered(m):  Eq. eq_Fornberg_centered (Sec. 4.1).
* k_staggered / k_centered: Eqs. staggered_modified_wave_number /
  centered_modified_wave_number (Sec. 4.1); order 0 means infinite spectral
  order, where both reduce to k (App. C).
* zeta: the Fourier symbol of finite-order centering (App. C, Eq. for zeta_F).

Coefficients are exact rationals (fractions.Fraction); trigonometric factors
are evaluated with an exact integer reduction of the angle so that the special
points (k = 0, Nyquist) give exact zeros and ones.
"""
from fractions import Fraction
from math import factorial

import numpy as np


def alpha_staggered(m):
    """Staggered Fornberg coefficients alpha^s_{m,n}, n = 1..m (Eq. eq_Fornberg_staggered).

    alpha^s_{m,n} = (-1)^{n+1} [(2m)! / (2^{2m} m!)]^2 * 4 / ((2n-1) (m-n)! (m+n-1)!)
    """
    pref = Fraction(factorial(2 * m), 2 ** (2 * m) * factorial(m)) ** 2
    return [(-1) ** (n + 1) * pref * Fraction(4, (2 * n - 1) * factorial(m - n) * factorial(m + n - 1))
            for n in range(1, m + 1)]


def alpha_centered(m):
    """Centered Fornberg coefficients alpha^c_{m,n}, n = 1..m (Eq. eq_Fornberg_centered).

    alpha^c_{m,n} = (-1)^{n+1} 2 (m!)^2 / ((m-n)! (m+n)!)
    """
    return [(-1) ** (n + 1) * Fraction(2 * factorial(m) ** 2, factorial(m - n) * factorial(m + n))
            for n in range(1, m + 1)]


def to_longdouble(q):
    """Correctly rounded np.longdouble value of a Fraction (decimal string route)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    return np.longdouble(str(Decimal(q.numerator) / Decimal(q.denominator)))


def signed_index(N):
    """Signed DFT indices for an axis of N points: 0..N/2-1, then -N/2..-1.

    The Nyquist index N/2 is taken as -N/2 (k = -pi/dx).
    """
    j = np.arange(N)
    return np.where(j < N // 2, j, j - N)


def wave_numbers(N, dx):
    """k_j = 2 pi m_j / (N dx) for the signed indices m_j (App. A.1, Eq. Fourier_discrete)."""
    return 2.0 * np.pi * signed_index(N) / (N * dx)


_PI_LD = np.longdouble("3.14159265358979323846264338327950288")


def _sin_pi_frac(p, q):
    """sin(pi p / q) in long double for integer arrays p and integer q > 0.

    The angle is reduced modulo 2 pi on integers and folded into [0, pi/2] so
    that multiples of pi/2 give exact 0 or +-1.
    """
    p = np.asarray(p, dtype=np.int64) % (2 * q)          # angle in [0, 2 pi)
    sign = np.where(p >= q, -1, 1)                        # sin(x + pi) = -sin(x)
    p = np.where(p >= q, p - q, p)                        # angle in [0, pi)
    p = np.where(2 * p > q, q - p, p)                     # sin(pi - x) = sin(x): angle in [0, pi/2]
    val = np.sin(p.astype(np.longdouble) * _PI_LD / np.longdouble(q))
    val = np.where(2 * p == q, np.longdouble(1), val)
    val = np.where(p == 0, np.longdouble(0), val)
    return sign * val


def sin_pi_frac(p, q):
    """sin(pi p / q) in long double with exact special values (see _sin_pi_frac)."""
    return _sin_pi_frac(p, q)


def cos_pi_frac(p, q):
    """cos(pi p / q) = sin(pi (p + q/2) / q), computed as sin(pi (2p + q) / (2q))."""
    return _sin_pi_frac(2 * np.asarray(p, dtype=np.int64) + q, 2 * q)


def k_staggered(N, dx, order):
    """[k]_s for the N signed wave numbers of an axis (Eq. staggered_modified_wave_number).

    [k]_s = sum_n alpha^s_{m,n} sin(k (n - 1/2) dx) / ((n - 1/2) dx), with 2m = order.
    k (n - 1/2) dx = pi j (2n - 1) / N for signed index j.  order 0 -> k itself.
    Returned in long double.
    """
    j = signed_index(N)
    dxl = np.longdouble(dx)
    if order == 0:
        return 2 * _PI_LD * j.astype(np.longdouble) / (N * dxl)
    m = order // 2
    out = np.zeros(N, dtype=np.longdouble)
    for n, a in enumerate(alpha_staggered(m), start=1):
        out += to_longdouble(a) * sin_pi_frac(j * (2 * n - 1), N) / ((n - np.longdouble(0.5)) * dxl)
    return out


def k_centered(N, dx, order):
    """[k]_c for the N signed wave numbers of an axis (Eq. centered_modified_wave_number).

    [k]_c = sum_n alpha^c_{m,n} sin(k n dx) / (n dx); k n dx = 2 pi j n / N.
    order 0 -> k itself.  Returned in long double.
    """
    j = signed_index(N)
    dxl = np.longdouble(dx)
    if order == 0:
        return 2 * _PI_LD * j.astype(np.longdouble) / (N * dxl)
    m = order // 2
    out = np.zeros(N, dtype=np.longdouble)
    for n, a in enumerate(alpha_centered(m), start=1):
        out += to_longdouble(a) * sin_pi_frac(2 * j * n, N) / (n * dxl)
    return out


def zeta(N, order):
    """Centering symbol zeta = sum_n alpha^s_{m,n} cos(k (n - 1/2) dx) (App. C).

    Multiplies the (paper-convention) spectrum of a quantity centered once along
    an axis, in either direction (nodal -> staggered or staggered -> nodal).
    Returned in long double for the N signed wave numbers of the axis.
    """
    j = signed_index(N)
    m = order // 2
    out = np.zeros(N, dtype=np.longdouble)
    for n, a in enumerate(alpha_staggered(m), start=1):
        out += to_longdouble(a) * cos_pi_frac(j * (2 * n - 1), N)
    return out
