"""Pins for oracle.grid: finite-order centering stencils and Fourier conventions.

Checked against: the centering's Fourier symbol zeta (App. C) on single grid
modes, polynomial exactness on an aperiodic patch, the convergence order on
cos^5(4 pi x) (the test function of Sec. 3, Fig. 4), the transpose relation of
the two centering directions, and brute-force direct DFT sums with the
paper's position-dependent phase (App. A.1).
"""
import numpy as np
import pytest

from oracle import fornberg, grid


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_centering_on_single_mode_is_zeta(order):
    N = 32
    z = fornberg.zeta(N, order).astype(float)
    j = np.arange(N)
    for m in (1, 3, 7, 12, 16):
        k = 2 * np.pi * fornberg.signed_index(N)[m] / N
        phase = 0.37
        stag = np.cos(k * (j + 0.5) + phase)              # a mode sampled at the cell centres
        nod = grid.center_staggered_to_nodal_1d(stag, 0, order)
        np.testing.assert_allclose(nod, z[m] * np.cos(k * j + phase), atol=1e-14)
        back = grid.center_nodal_to_staggered_1d(np.cos(k * j + phase), 0, order)
        np.testing.assert_allclose(back, z[m] * np.cos(k * (j + 0.5) + phase), atol=1e-14)


@pytest.mark.parametrize("m", [1, 2, 4])
def test_centering_exact_on_polynomials(m):
    # interpolation at order 2m reproduces polynomials of degree <= 2m-1 away from the wrap
    N = 64
    x_c = np.arange(N) + 0.5
    for deg in range(2 * m):
        p = np.polynomial.Polynomial(np.random.default_rng(deg).normal(size=deg + 1))
        nod = grid.center_staggered_to_nodal_1d(p(x_c / N), 0, 2 * m)
        inner = slice(m + 1, N - m - 1)
        np.testing.assert_allclose(nod[inner], p(np.arange(N) / N)[inner], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_centering_convergence_order_cos5(m):
    # Sec. 3: cos^5(4 pi x) on [0,1) interpolated at order 2m; the error falls as dx^{2m}
    # (the k = m moment of alpha^s does not vanish, so not dx^{2m+2}).
    f = lambda x: np.cos(4 * np.pi * x) ** 5
    errs = []
    for N in (64, 128, 256):
        x = np.arange(N) / N
        nod = grid.center_staggered_to_nodal_1d(f(x + 0.5 / N), 0, 2 * m)
        errs.append(np.max(np.abs(nod - f(x))))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - 2 * m) < 0.15


def test_centering_directions_are_transposes():
    N, order = 12, 8
    eye = np.eye(N)
    A = np.stack([grid.center_staggered_to_nodal_1d(eye[:, i], 0, order) for i in range(N)], axis=1)
    B = np.stack([grid.center_nodal_to_staggered_1d(eye[:, i], 0, order) for i in range(N)], axis=1)
    np.testing.assert_allclose(A.T, B, atol=1e-16)


@pytest.mark.parametrize("name", list(grid.STAG))
def test_spectral_convention_matches_direct_sum(name):
    shape, dx = (4, 2, 8), (0.5, 1.5, 0.25)
    rng = np.random.default_rng(7)
    f = rng.normal(size=shape)
    X, Y, Z = grid.positions(shape, dx, name)
    k = [fornberg.wave_numbers(shape[a], dx[a]) for a in range(3)]
    direct = np.zeros(shape, dtype=complex)
    for a in range(shape[0]):
        for b in range(shape[1]):
            for c in range(shape[2]):
                direct[a, b, c] = np.sum(f * np.exp(-1j * (k[0][a] * X + k[1][b] * Y + k[2][c] * Z)))
    np.testing.assert_allclose(grid.to_spectral(f, name, dx), direct, atol=1e-12)
    back, im = grid.from_spectral(grid.to_spectral(f, name, dx), name, dx)
    np.testing.assert_allclose(back, f, atol=1e-14)
    assert im < 1e-14


def test_fft_matches_direct_dft_and_parseval():
    shape = (4, 8, 2)
    rng = np.random.default_rng(3)
    f = rng.normal(size=shape)
    idx = [np.arange(n) for n in shape]
    F = np.zeros(shape, dtype=complex)
    for a in range(shape[0]):
        for b in range(shape[1]):
            for c in range(shape[2]):
                ph = np.exp(-2j * np.pi * (a * idx[0][:, None, None] / shape[0]
                                           + b * idx[1][None, :, None] / shape[1]
                                           + c * idx[2][None, None, :] / shape[2]))
                F[a, b, c] = np.sum(f * ph)
    np.testing.assert_allclose(np.fft.fftn(f), F, atol=1e-13)
    assert abs(np.sum(f ** 2) - np.sum(np.abs(F) ** 2) / f.size) < 1e-12


def test_bilinear_filter_symbol_sum_and_stencil():
    from oracle import grid, fornberg
    shape = (8, 6, 16)
    # on a single Fourier mode the filter multiplies by prod_a cos^2(k_a dx_a / 2) per pass
    rng = np.random.default_rng(2)
    m = (3, 1, 5)
    idx = np.indices(shape)
    phase = sum(2 * np.pi * m[a] * idx[a] / shape[a] for a in range(3))
    f = np.cos(phase)
    for passes in (1, 2):
        sym = np.prod([np.cos(np.pi * m[a] / shape[a]) ** 2 for a in range(3)]) ** passes
        np.testing.assert_allclose(grid.bilinear_filter(f, passes), sym * f, atol=1e-14)
    # the sum over the grid is unchanged
    g = rng.normal(size=shape)
    assert abs(grid.bilinear_filter(g, 3).sum() - g.sum()) < 1e-12
    # a delta becomes the outer product of (1/4, 1/2, 1/4)
    d = np.zeros(shape)
    d[4, 3, 8] = 1.0
    h = grid.bilinear_filter(d, 1)
    w = np.array([0.25, 0.5, 0.25])
    ref = np.zeros(shape)
    ref[3:6, 2:5, 7:10] = w[:, None, None] * w[None, :, None] * w[None, None, :]
    np.testing.assert_allclose(h, ref, atol=1e-16)
    del fornberg
