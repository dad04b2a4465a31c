"""Pins of the oracle's diagnostics (stencil extent, beam RMS, vacuum dispersion)
against closed forms and explicit sums."""
import numpy as np

from oracle import diagnostics, fornberg, psatd


def _m(N):
    return fornberg.signed_index(N)


def test_stencil_extent_of_one_is_a_delta():
    g = np.ones((8, 6, 4))
    for axis in range(3):
        G = diagnostics.stencil_extent(g, axis)
        ref = np.zeros(g.shape[axis])
        ref[0] = 1.0
        np.testing.assert_allclose(G, ref, atol=1e-15)


def test_stencil_extent_of_a_cosine_is_two_half_spikes():
    # g = cos(k_x dx) on the integer grid is the stencil (f_{j-1} + f_{j+1}) / 2
    N = 16
    kx = 2 * np.pi * _m(N) / N
    g = np.broadcast_to(np.cos(kx)[:, None, None], (N, 4, 8))
    G = diagnostics.stencil_extent(g, 0)
    ref = np.zeros(N)
    ref[1] = ref[N - 1] = 0.5
    np.testing.assert_allclose(G, ref, atol=1e-15)


def test_stencil_extent_of_a_separable_quantity_by_explicit_sums():
    rng = np.random.default_rng(3)
    shape = (6, 5, 4)
    a = rng.normal(size=6) + 1j * rng.normal(size=6)
    b = rng.normal(size=5) + 1j * rng.normal(size=5)
    c = rng.normal(size=4) + 1j * rng.normal(size=4)
    g = a[:, None, None] * b[None, :, None] * c[None, None, :]
    G = diagnostics.stencil_extent(g, 1)
    ref = np.zeros(5)
    for j in range(5):
        s = 0j
        for m in range(5):
            s += b[m] * np.exp(2j * np.pi * m * j / 5)
        ref[j] = abs(s / 5) * abs(np.mean(a)) * abs(np.mean(c))
    np.testing.assert_allclose(G, ref, rtol=1e-13, atol=1e-15)


def test_beam_rms_closed_forms():
    a, b = 0.3, 1.7
    # four particles at (+-a, 0), (0, +-b)... RMS per axis over all particles
    x = np.array([-a, a])
    y = np.array([-b, b])
    assert abs(diagnostics.beam_rms(x, y, np.ones(2)) - 0.5 * (a + b)) < 1e-15
    # two weights: sigma = |x1 - x2| sqrt(w1 w2) / (w1 + w2)
    w = np.array([1.0, 3.0])
    x = np.array([2.0, 5.0])
    y = np.array([-1.0, 1.0])
    sx = 3.0 * np.sqrt(3.0) / 4.0
    sy = 2.0 * np.sqrt(3.0) / 4.0
    assert abs(diagnostics.beam_rms(x, y, w) - 0.5 * (sx + sy)) < 1e-14
    # invariant under translation, scales linearly
    rng = np.random.default_rng(1)
    x, y, w = rng.normal(size=100), rng.normal(size=100), rng.uniform(0.5, 2, 100)
    d = diagnostics.beam_rms(x, y, w)
    assert abs(diagnostics.beam_rms(x + 7.0, y - 3.0, w) - d) < 1e-12
    assert abs(diagnostics.beam_rms(2 * x, 2 * y, w) - 2 * d) < 1e-12


def _dispersion(shape, dx, dt, order, v=(0.0, 0.0, 0.0), axis=2):
    co = psatd.coefficients(shape, dx, dt, order, v)
    k = psatd.staggered_k_grid(shape, dx, order)
    return diagnostics.vacuum_dispersion(co, k, axis, 1.0, dt)


def test_vacuum_dispersion_standard_closed_forms():
    shape, dx, dt = (4, 4, 32), (1.0, 1.0, 1.0), 0.5
    N = shape[2]
    k = 2 * np.pi * _m(N) / N
    # infinite order: omega = c |k|
    w = _dispersion(shape, dx, dt, (0, 0, 0))
    np.testing.assert_allclose(w, np.abs(k), rtol=1e-12, atol=1e-13)
    # order 2: [k]_s = 2 sin(k dx / 2) / dx
    w = _dispersion(shape, dx, dt, (2, 2, 2))
    np.testing.assert_allclose(w, np.abs(2 * np.sin(k / 2)), rtol=1e-12, atol=1e-13)


def test_vacuum_dispersion_galilean_phases():
    shape, dx, dt = (4, 4, 32), (1.0, 1.0, 1.0), 0.5
    v = (0.0, 0.0, 0.6)
    order = (8, 8, 8)
    N = shape[2]
    ks = np.asarray(fornberg.k_staggered(N, 1.0, 8), dtype=np.float64)
    kc = np.asarray(fornberg.k_centered(N, 1.0, 8), dtype=np.float64)
    w = _dispersion(shape, dx, dt, order, v)
    # eigenvalues theta^2 exp(+-i omega_s dt), theta^2 = exp(i Omega_c dt)
    ph = np.stack([v[2] * kc * dt + np.abs(ks) * dt, v[2] * kc * dt - np.abs(ks) * dt])
    ph = np.angle(np.exp(1j * ph))
    np.testing.assert_allclose(w, np.max(ph, axis=0) / dt, rtol=1e-11, atol=1e-12)


def test_field_energy_uniform_fields_closed_form():
    """W = 1/2 (eps0 |E|^2 + |B|^2 / mu0) V with mu0 = 1 / (eps0 c^2), for uniform fields and
    c, eps0 different from 1."""
    shape, dx, c, eps0 = (4, 6, 8), (0.5, 0.25, 2.0), 3.0, 0.7
    E = [np.full(shape, 1.5), np.zeros(shape), np.full(shape, -2.0)]
    B = [np.zeros(shape), np.full(shape, 0.5), np.zeros(shape)]
    V = np.prod(shape) * np.prod(dx)
    want = 0.5 * (eps0 * (1.5 ** 2 + 2.0 ** 2) + 0.5 ** 2 * eps0 * c * c) * V
    assert abs(diagnostics.field_energy(E, B, dx, c=c, eps0=eps0) - want) < 1e-13 * want
    # a box: the same density over its volume
    lo, hi = (1, 2, 3), (3, 5, 8)
    Vb = np.prod([hi[a] - lo[a] for a in range(3)]) * np.prod(dx)
    wb = diagnostics.field_energy(E, B, dx, c=c, eps0=eps0, box_lo=lo, box_hi=hi)
    assert abs(wb - want * Vb / V) < 1e-13 * want
