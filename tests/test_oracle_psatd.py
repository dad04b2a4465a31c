"""Pins for oracle.psatd: the PSATD update coefficients and k-space updates.

The main pin is independent of the paper's closed forms: for a single mode,
the Fourier-space Maxwell system of App. A (Eqs. eq_Faraday_Fourier,
eq_AmpereMaxwell_Fourier, Galilean form) with J constant over the step is a
linear ODE with constant forcing, solved exactly by the matrix exponential of
the augmented system (scipy.linalg.expm).  rho^n and rho^{n+1} follow from
Gauss's law at t^n and t^{n+1}.  The averaged fields are the time average of
that exact solution over [t^{n+1/2}, t^{n+3/2}] (Gauss-Legendre quadrature).
Further pins: the vacuum dispersion relations of App. B on a real-space
plane wave, electrostatic equilibrium, the k = 0 limits, and the
v_gal -> 0 limit of Sec. 4.3.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import fornberg, grid, psatd


def _exact_mode(ks, Om, E0, B0, J, t, c=1.0, eps0=1.0):
    """Exact E(t), B(t) of dB/dt = i Om B - i ks x E, dE/dt = i Om E + i c^2 ks x B - J/eps0."""
    def crossmat(k):
        return np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]], dtype=complex)
    K = crossmat(ks)
    A = np.zeros((7, 7), dtype=complex)
    A[0:3, 0:3] = 1j * Om * np.eye(3)
    A[0:3, 3:6] = 1j * c * c * K
    A[0:3, 6] = -J / eps0
    A[3:6, 3:6] = 1j * Om * np.eye(3)
    A[3:6, 0:3] = -1j * K
    y0 = np.concatenate([E0, B0, [1.0]])
    y = expm(A * t) @ y0
    return y[0:3], y[3:6]


def _random_mode_state(rng, ks):
    E0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    B0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    if np.linalg.norm(ks) > 0:
        kh = ks / np.linalg.norm(ks)
        B0 = B0 - kh * np.dot(kh, B0)           # magnetic Gauss law: [k]_s . B = 0
    J = rng.normal(size=3) + 1j * rng.normal(size=3)
    return E0, B0, J


def _coeff_at(shape, dx, dt, order, v_gal, idx, averaged, c=1.0, eps0=1.0):
    co = psatd.coefficients(shape, dx, dt, order, v_gal, c, eps0, averaged=averaged)
    ks, kc = psatd.modified_wave_vectors(shape, dx, order)
    ksv = np.array([float(ks[a][idx[a]]) for a in range(3)])
    kcv = np.array([float(kc[a][idx[a]]) for a in range(3)])
    return {k: v[idx] for k, v in co.items()}, ksv, kcv


CASES = [
    # shape, dx, dt, spectral order, v_gal, mode index
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (0, 0, 0), (0, 0, 0), (1, 2, 3)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (0, 0, 0), (0, 0, 0), (4, 4, 8)),
    ((8, 8, 16), (0.2, 0.2, 0.04), 0.04, (0, 0, 0), (0, 0, 0), (1, 0, 1)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (16, 16, 16), (0, 0, 0.995), (1, 2, 3)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (16, 16, 16), (0, 0, 0.995), (0, 0, 1)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (8, 8, 8), (0.1, -0.2, 0.7), (3, 6, 13)),
    ((8, 8, 32), (0.1, 0.1, 0.02), 0.02, (16, 16, 16), (0, 0, np.sqrt(1 - 1e-6)), (1, 1, 2)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (16, 16, 16), (0, 0, 0.9), (2, 1, 0)),
    ((8, 8, 16), (1.0, 1.0, 1.0), 1.0, (0, 0, 0), (0, 0, 0), (0, 0, 0)),
]


@pytest.mark.parametrize("case", CASES)
def test_update_matches_exact_ode_solution(case):
    shape, dx, dt, order, v_gal, idx = case
    for c, eps0 in [(1.0, 1.0), (2.0, 0.5)]:
        co, ksv, kcv = _coeff_at(shape, dx, dt, order, v_gal, idx, True, c, eps0)
        Om = float(np.dot(v_gal, kcv))
        rng = np.random.default_rng(11)
        E0, B0, J = _random_mode_state(rng, ksv)
        rho_n = 1j * eps0 * np.dot(ksv, E0)                      # Gauss: [k]_s . E = -i rho / eps0
        E1, B1 = _exact_mode(ksv, Om, E0, B0, J, dt, c, eps0)
        rho_np1 = 1j * eps0 * np.dot(ksv, E1)
        wrap = lambda v: [np.array(x) for x in v]
        En, Bn = psatd.update(wrap(E0), wrap(B0), wrap(J), rho_n, rho_np1, co, list(ksv), c)
        scale = max(np.abs(E1).max(), c * np.abs(B1).max())
        np.testing.assert_allclose(np.array(En), E1, atol=1e-12 * scale)
        np.testing.assert_allclose(c * np.array(Bn), c * B1, atol=1e-12 * scale)
        # averaged fields: (1/dt) * integral over [dt/2, 3 dt/2] of the exact solution
        xg, wg = np.polynomial.legendre.leggauss(24)
        tq = dt + 0.5 * dt * xg
        Ea = sum(0.5 * w * _exact_mode(ksv, Om, E0, B0, J, t, c, eps0)[0] for t, w in zip(tq, wg))
        Ba = sum(0.5 * w * _exact_mode(ksv, Om, E0, B0, J, t, c, eps0)[1] for t, w in zip(tq, wg))
        Eav, Bav = psatd.update_averaged(wrap(E0), wrap(B0), wrap(J), rho_n, rho_np1, co, list(ksv), c)
        np.testing.assert_allclose(np.array(Eav), Ea, atol=1e-12 * scale)
        np.testing.assert_allclose(c * np.array(Bav), c * Ba, atol=1e-12 * scale)


def test_k0_limits():
    co = psatd.coefficients((4, 4, 4), (1.0, 1.0, 1.0), 0.5, (0, 0, 0), averaged=True, eps0=2.0)
    d = {k: v[0, 0, 0] for k, v in co.items()}
    assert d["TC"] == 1 and d["TS"] == 0.5 and d["X4"] == -0.25
    assert abs(d["Psi1"] - 1) == 0 and d["Psi2"] == -0.5 and d["Y4"] == -0.25


def test_galilean_tends_to_standard():
    shape, dx, dt = (8, 8, 16), (1.0, 1.0, 1.0), 1.0
    std = psatd.coefficients(shape, dx, dt, (16, 16, 16))
    for v, tol in [(1e-3, 5e-3), (1e-6, 5e-6)]:
        gal = psatd.coefficients(shape, dx, dt, (16, 16, 16), v_gal=(0, 0, v))
        for k in std:
            assert np.max(np.abs(gal[k] - std[k])) < tol, k


def _plane_wave_fields(shape, dx, kvec, omega, t, c=1.0):
    """Transverse plane wave along z (E_y, B_x = -E_y/c), sampled at each Yee position."""
    E = [np.zeros(shape) for _ in range(3)]
    B = [np.zeros(shape) for _ in range(3)]
    X, Y, Z = grid.positions(shape, dx, "Ey")
    E[1] = np.cos(kvec * Z - omega * t)
    X, Y, Z = grid.positions(shape, dx, "Bx")
    B[0] = -np.cos(kvec * Z - omega * t) / c
    return E, B


@pytest.mark.parametrize("order,v", [(0, 0.0), (16, 0.0), (16, 0.9), (4, -0.5)])
def test_vacuum_plane_wave_dispersion(order, v):
    # App. B: omega = c [k]_s + v_gal (k - [k]_c); in Galilean coordinates the mode advances
    # by (omega - v_gal k) dt = (c [k]_s - v_gal [k]_c) dt per step.
    shape, dx, dt, nsteps = (4, 4, 32), (1.0, 1.0, 0.5), 0.4, 25
    m = 5
    kz = 2 * np.pi * m / (shape[2] * dx[2])
    ks = float(fornberg.k_staggered(shape[2], dx[2], order)[m])
    kc = float(fornberg.k_centered(shape[2], dx[2], order)[m])
    if order == 0:
        assert ks == pytest.approx(kz, rel=1e-15)
    rate = ks - v * kc                                       # c = 1
    variant = (0, 0, v)
    co = psatd.coefficients(shape, dx, dt, (order,) * 3, variant)
    kg = psatd.staggered_k_grid(shape, dx, (order,) * 3)
    E, B = _plane_wave_fields(shape, dx, kz, 0.0, 0.0)
    Z = [np.zeros(shape) for _ in range(3)]
    for _ in range(nsteps):
        Eh = [grid.to_spectral(E[a], grid.E_NAMES[a], dx) for a in range(3)]
        Bh = [grid.to_spectral(B[a], grid.B_NAMES[a], dx) for a in range(3)]
        Jh = [grid.to_spectral(Z[a], grid.J_NAMES[a], dx) for a in range(3)]
        r = grid.to_spectral(Z[0], "rho", dx)
        En, Bn = psatd.update(Eh, Bh, Jh, r, r, co, kg)
        E = [grid.from_spectral(En[a], grid.E_NAMES[a], dx)[0] for a in range(3)]
        B = [grid.from_spectral(Bn[a], grid.B_NAMES[a], dx)[0] for a in range(3)]
    Ee, Be = _plane_wave_fields(shape, dx, kz, rate, nsteps * dt)
    for a in range(3):
        np.testing.assert_allclose(E[a], Ee[a], atol=1e-12)
        np.testing.assert_allclose(B[a], Be[a], atol=1e-12)


def test_electrostatic_equilibrium():
    # J = 0, rho^n = rho^{n+1} = rho, E longitudinal from Gauss's law: one update returns E.
    shape, dx, dt = (8, 8, 8), (1.0, 0.7, 1.3), 0.6
    rng = np.random.default_rng(5)
    rho = rng.normal(size=shape)
    rh = grid.to_spectral(rho, "rho", dx)
    for order in [(0, 0, 0), (8, 8, 8)]:
        co = psatd.coefficients(shape, dx, dt, order)
        k = psatd.staggered_k_grid(shape, dx, order)
        k2 = sum(k[a] ** 2 for a in range(3))
        k2s = np.where(k2 == 0, 1.0, k2)
        EL = [np.where(k2 == 0, 0, -1j * rh * k[a] / k2s) for a in range(3)]
        Z = [np.zeros(shape, dtype=complex) for _ in range(3)]
        En, Bn = psatd.update(EL, Z, Z, rh, rh, co, k)
        # the modes where [k]_s = 0 other than k = 0 (none here) carry no longitudinal field
        for a in range(3):
            np.testing.assert_allclose(En[a], EL[a], atol=1e-12 * np.abs(EL[a]).max())
            np.testing.assert_allclose(Bn[a], 0, atol=1e-12)
