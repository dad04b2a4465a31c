"""Pins of the FDTD solver of the hybrid FDTD cycle (oracle/fdtd.py).

Textbook facts checked: Yee's difference and the fourth-order staggered stencil (9/8, -1/24),
exactness on polynomials of degree <= 2m, the symbol of a sampled Fourier mode, div curl = 0 on
the Yee grid (so div B stays 0 and Gauss's law changes only by -dt div J / eps0), the Yee vacuum
dispersion relation sin(omega dt / 2) = c dt [k]_s / 2 with unit-modulus eigenvalues, the Courant
limit, and agreement with the PSATD update of the same spatial order as dt -> 0 (leapfrog local
error O(dt^3))."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fdtd, fornberg, grid, psatd, step


def test_weights_textbook():
    assert fdtd.fd_weights(2, 1.0) == [1.0]
    w = fdtd.fd_weights(4, 0.5)
    assert w == [float(Fraction(9, 8)) / 0.5, float(Fraction(-1, 24)) / 0.5]


def _mode_k(N, dx, order, j):
    k = 2 * np.pi * j / (N * dx)
    if order == 2:
        return 2 * np.sin(k * dx / 2) / dx
    if order == 4:
        return (9 / 8 * 2 * np.sin(k * dx / 2) - 1 / 24 * 2 * np.sin(3 * k * dx / 2)) / dx
    return float(fornberg.k_staggered(N, dx, order)[j])


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_derivative_of_a_mode(order, axis):
    shape, dx = [16, 16, 16], 0.3
    N, j = shape[axis], 3
    k = 2 * np.pi * j / (N * dx)
    x = np.arange(N) * dx
    bs = [1, 1, 1]
    bs[axis] = N
    f = np.broadcast_to(np.cos(k * x).reshape(bs), shape).copy()
    K = _mode_k(N, dx, order, j)
    d = fdtd.d_to_half(f, axis, order, dx)
    want = np.broadcast_to((-K * np.sin(k * (x + dx / 2))).reshape(bs), shape)
    assert np.max(np.abs(d - want)) < 1e-13 * abs(K)
    s = np.broadcast_to(np.cos(k * (x + dx / 2)).reshape(bs), shape).copy()
    d = fdtd.d_to_node(s, axis, order, dx)
    want = np.broadcast_to((-K * np.sin(k * x)).reshape(bs), shape)
    assert np.max(np.abs(d - want)) < 1e-13 * abs(K)
    # the symbol tends to k for smooth modes
    if order == 8:
        assert abs(K - k) < 5e-4 * k   # k dx = 1.18 here


@pytest.mark.parametrize("order", [2, 4, 6])
def test_exact_on_polynomials(order):
    """The order-2m staggered difference differentiates polynomials of degree <= 2m exactly."""
    N, dx, m = 64, 1.0 / 64, order // 2
    x = np.arange(N) * dx
    p = 2 * m
    f = ((x - 0.5) ** p)[:, None, None] * np.ones((1, 2, 2))
    d = fdtd.d_to_half(f, 0, order, dx)[:, 0, 0]
    xh = x + dx / 2
    want = p * (xh - 0.5) ** (p - 1)
    inner = slice(m, N - m)          # away from the periodic wrap
    assert np.max(np.abs(d[inner] - want[inner])) < 1e-12
    s = ((xh - 0.5) ** p)[:, None, None] * np.ones((1, 2, 2))
    d = fdtd.d_to_node(s, 0, order, dx)[:, 0, 0]
    want = p * (x - 0.5) ** (p - 1)
    assert np.max(np.abs(d[inner] - want[inner])) < 1e-12
    # one degree more is not exact
    f = ((x - 0.5) ** (p + 1))[:, None, None] * np.ones((1, 2, 2))
    d = fdtd.d_to_half(f, 0, order, dx)[:, 0, 0]
    assert np.max(np.abs(d[inner] - (p + 1) * (xh[inner] - 0.5) ** p)) > 1e-11


@pytest.mark.parametrize("orders", [(2, 2, 2), (4, 2, 8), (8, 8, 16)])
def test_div_curl_zero_and_gauss(orders):
    rng = np.random.default_rng(7)
    shape, dx = (8, 16, 32), (0.7, 1.1, 0.4)
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    J = [rng.normal(size=shape) for _ in range(3)]
    assert np.max(np.abs(fdtd.div_B(fdtd.curl_E(E, orders, dx), orders, dx))) < 1e-12 * 50
    assert np.max(np.abs(fdtd.div_E(fdtd.curl_B(B, orders, dx), orders, dx))) < 1e-12 * 50
    dt, c, eps0 = 0.1, 1.3, 0.8
    En, Bn = fdtd.yee_update(E, B, J, dt, orders, dx, c, eps0)
    lhs = fdtd.div_E(En, orders, dx) - fdtd.div_E(E, orders, dx)
    rhs = -dt / eps0 * fdtd.div_E(J, orders, dx)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * 50
    assert np.max(np.abs(fdtd.div_B(Bn, orders, dx) - fdtd.div_B(B, orders, dx))) < 1e-12 * 50


@pytest.mark.parametrize("order,j,cdt", [(2, 1, 0.5), (2, 7, 0.9), (4, 5, 0.6), (8, 3, 0.4)])
def test_vacuum_dispersion_yee(order, j, cdt):
    """E^x(z), B^y(z) plane wave: the one-step map has eigenvalues exp(+-i omega dt) with
    sin(omega dt / 2) = c dt [k]_s / 2 (Yee's dispersion relation, order 2m symbol)."""
    shape, dz, c = (2, 2, 16), 1.0, 1.5
    dt = cdt * dz / c
    N = shape[2]
    k = 2 * np.pi * j / (N * dz)
    z = np.arange(N) * dz
    cosn = np.cos(k * z)[None, None, :] * np.ones(shape)          # E^x: nodal along z
    sinh = np.sin(k * (z + dz / 2))[None, None, :] * np.ones(shape)  # B^y: staggered along z
    orders = (2, 2, order)
    Z = np.zeros(shape)

    def one(a, b):
        En, Bn = fdtd.yee_update([a * cosn, Z, Z], [Z, b * sinh, Z], [Z, Z, Z], dt, orders,
                                 (1.0, 1.0, dz), c)
        return (np.sum(En[0] * cosn) / np.sum(cosn * cosn), np.sum(Bn[1] * sinh) / np.sum(sinh * sinh))

    M = np.array([one(1.0, 0.0), one(0.0, 1.0)]).T
    lam = np.linalg.eigvals(M)
    assert np.allclose(np.abs(lam), 1.0, atol=1e-13)
    K = _mode_k(N, dz, order, j)
    want = 2 * np.arcsin(c * dt * K / 2)
    assert np.allclose(np.sort(np.abs(np.angle(lam))), [want, want], atol=1e-13)


def test_courant_limit():
    assert abs(fdtd.courant_limit((2, 2, 2), (1.0, 1.0, 1.0)) - 1 / np.sqrt(3)) < 1e-15
    dx = (0.2, 0.2, 0.04)
    want = 1 / (2.0 * np.sqrt(sum(1 / d ** 2 for d in dx)))
    assert abs(fdtd.courant_limit((2, 2, 2), dx, c=2.0) - want) < 1e-15 * want
    # the Nyquist mode of the diagonal direction grows just above the limit, not below it
    for f, grows in [(0.99, False), (1.01, True)]:
        dt = f * fdtd.courant_limit((2, 2, 2), (1.0, 1.0, 1.0))
        shape = (4, 4, 4)
        rng = np.random.default_rng(3)
        E = [rng.normal(size=shape) * 1e-3 for _ in range(3)]
        B = [np.zeros(shape) for _ in range(3)]
        Z = [np.zeros(shape) for _ in range(3)]
        for _ in range(400):
            E, B = fdtd.yee_update(E, B, Z, dt, (2, 2, 2), (1.0, 1.0, 1.0))
        amp = max(np.abs(e).max() for e in E)
        assert (amp > 1.0) == grows


def test_agrees_with_psatd_as_dt_shrinks():
    """FDTD and the PSATD update with the same order-2m [k]_s solve the same semi-discrete
    system; the leapfrog step differs from the exact one by O(dt^3)."""
    shape, dx, orders = (8, 8, 16), (1.0, 1.0, 0.5), (4, 4, 4)
    rng = np.random.default_rng(5)
    k = psatd.staggered_k_grid(shape, dx, orders)
    k2 = sum(k[a] ** 2 for a in range(3))
    k2s = np.where(k2 == 0, 1.0, k2)

    def solenoidal(names, smooth):
        F = [grid.to_spectral(rng.normal(size=shape), n, dx) * smooth for n in names]
        kd = sum(k[a] * F[a] for a in range(3)) / k2s
        return [grid.from_spectral(F[a] - k[a] * kd, names[a], dx)[0] for a in range(3)]

    smooth = np.exp(-0.5 * k2.real if np.iscomplexobj(k2) else -0.5 * k2)
    E0, B0 = solenoidal(grid.E_NAMES, smooth), solenoidal(grid.B_NAMES, smooth)
    Z = [np.zeros(shape) for _ in range(3)]
    errs = []
    for dt in (0.08, 0.04):
        p = step.Params(shape, dx, dt, 1, (2, 2, 2), spectral_order=orders)
        Ep, Bp, _, _ = step.maxwell_update(p, E0, B0, Z, np.zeros(shape), np.zeros(shape))
        Ef, Bf = fdtd.yee_update(E0, B0, Z, dt, orders, dx)
        errs.append(max(np.abs(Ef[a] - Ep[a]).max() for a in range(3)) +
                    max(np.abs(Bf[a] - Bp[a]).max() for a in range(3)))
    assert 7.0 < errs[0] / errs[1] < 9.0


def test_fdtd_cycle_charge_and_vacuum():
    """The hybrid FDTD cycle: with no particles it is yee_update; with particles, charge holds."""
    from paper_2106_12919_gb300 import workloads
    w = workloads.thermal_plasma(shape=(8, 8, 8), ppc=2)
    prm = dict(w["params"])
    prm.update(dt=0.4, cycle=step.HYBRID_FDTD, spectral_order=(0, 4, 2))
    p = step.Params(**prm)
    assert p.fd_orders() == (2, 4, 2)
    rng = np.random.default_rng(2)
    E = [rng.normal(size=p.shape) for _ in range(3)]
    B = [rng.normal(size=p.shape) for _ in range(3)]
    st = {"E": [e.copy() for e in E], "B": [b.copy() for b in B], "species": [], "rho": np.zeros(p.shape)}
    step.hybrid_step(p, st)
    Z = [np.zeros(p.shape) for _ in range(3)]
    En, Bn = fdtd.yee_update(E, B, Z, p.dt, p.fd_orders(), p.dx, p.c, p.eps0)
    for a in range(3):
        assert np.array_equal(st["E"][a], En[a]) and np.array_equal(st["B"][a], Bn[a])
    st = {"E": [np.zeros(p.shape) for _ in range(3)], "B": [np.zeros(p.shape) for _ in range(3)],
          "species": [dict(s) for s in w["species"]]}
    st["rho"] = step.initial_rho(p, st["species"])
    qtot = sum(float(np.sum(s["q"] * s["w"])) for s in st["species"])
    qabs = sum(float(np.sum(np.abs(s["q"] * s["w"]))) for s in st["species"])
    for _ in range(3):
        step.hybrid_step(p, st)
        assert abs(np.sum(st["rho"]) * np.prod(p.dx) - qtot) < 1e-12 * qabs
        assert all(np.all(np.isfinite(e)) for e in st["E"])


@pytest.mark.parametrize("order", [2, 4, 8, 16, 32])
def test_courant_bound_uses_the_largest_symbol(order):
    """The Courant limit takes [k]_s at the Nyquist wave number: the symbol is monotone on
    [0, pi/dx] (its derivative in k dx is the centering symbol zeta >= 0, App. C), so the
    Nyquist value is the maximum over every wave number of the grid."""
    N, dx = 64, 0.3
    ks = np.abs(fornberg.k_staggered(N, dx, order).astype(np.float64))
    ny = 2.0 * sum(w * (1 if n % 2 else -1) for n, w in enumerate(fdtd.fd_weights(order, dx), start=1))
    assert abs(ks.max() - ny) < 1e-12 * ny
    assert np.all(np.diff(ks[: N // 2 + 1]) > 0)        # signed indices 0..N/2-1, then the Nyquist -N/2
    assert np.all(fornberg.zeta(N, order)[: N // 2 + 1].astype(np.float64) >= -1e-15)
