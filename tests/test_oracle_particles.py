"""Pins for oracle.particles: B-spline shapes, gather, deposit, Boris push, tile bins.

Checked against: the Cox-de Boor recursion for centred B-splines (textbook,
independent of the closed forms), partition of unity and linear
reproduction, exact gathers of uniform/linear fields, gather/deposit
adjointness, total charge, the analytic gyration of the Boris rotation and
the exact pure-E kick, and a per-particle brute-force bin count.
"""
import numpy as np
import pytest

from oracle import particles


def _bspline(p, x):
    """Centred cardinal B-spline of degree p (support [-(p+1)/2, (p+1)/2]) by recursion."""
    if p == 0:
        return np.where((x >= -0.5) & (x < 0.5), 1.0, 0.0)
    return ((x + (p + 1) / 2) * _bspline(p - 1, x + 0.5) + ((p + 1) / 2 - x) * _bspline(p - 1, x - 0.5)) / p


@pytest.mark.parametrize("order", [1, 2, 3])
def test_shape_weights_are_bsplines(order):
    rng = np.random.default_rng(order)
    x = rng.uniform(0, 20, 2000)
    lo, w = particles.shape_weights(x, 1.0, order)
    assert w.shape == (order + 1, x.size)
    for n in range(order + 1):
        np.testing.assert_allclose(w[n], _bspline(order, x - (lo + n)), atol=1e-14)
    np.testing.assert_allclose(w.sum(axis=0), 1.0, atol=1e-14)                         # partition of unity
    np.testing.assert_allclose(sum((lo + n) * w[n] for n in range(order + 1)), x, atol=1e-12)  # first moment


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_uniform_and_linear_fields_exact(order):
    shape, dx = (16, 16, 16), (0.5, 1.0, 2.0)
    rng = np.random.default_rng(2)
    pos = [rng.uniform(4 * dx[a], 11 * dx[a], 500) for a in range(3)]
    X, Y, Z = np.meshgrid(*[np.arange(shape[a]) * dx[a] for a in range(3)], indexing="ij")
    const = np.full(shape, 3.25)
    lin = 0.3 * X - 1.1 * Y + 0.7 * Z + 2.0
    gc, gl = particles.gather([const, lin], pos, dx, order)
    np.testing.assert_allclose(gc, 3.25, atol=1e-13)
    np.testing.assert_allclose(gl, 0.3 * pos[0] - 1.1 * pos[1] + 0.7 * pos[2] + 2.0, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_deposit_gather_adjoint_and_charge(order):
    shape, dx = (8, 4, 8), (0.5, 1.0, 0.25)
    rng = np.random.default_rng(4)
    n = 3000
    pos = [rng.uniform(0, shape[a] * dx[a], n) for a in range(3)]
    v = rng.normal(size=n)
    F = rng.normal(size=shape)
    (rho,) = particles.deposit(shape, pos, [v], dx, order)
    dV = dx[0] * dx[1] * dx[2]
    (g,) = particles.gather([F], pos, dx, order)
    assert abs(np.sum(rho * F) * dV - np.sum(v * g)) < 1e-10 * np.sum(np.abs(v * g))
    assert abs(np.sum(rho) * dV - np.sum(v)) < 1e-11 * np.sum(np.abs(v))


def test_boris_pure_magnetic_gyration():
    # |u| conserved; rotation angle per step = 2 atan(q B dt / (2 m gamma)) about B
    q, m, dt, Bz = -1.0, 1.0, 0.3, 2.0
    u = [np.array([0.4]), np.array([0.0]), np.array([0.1])]
    gamma = np.sqrt(1 + 0.4 ** 2 + 0.1 ** 2)
    E = [np.zeros(1)] * 3
    B = [np.zeros(1), np.zeros(1), np.full(1, Bz)]
    un = particles.boris(u, E, B, q, m, dt)
    ang = np.arctan2(un[1][0], un[0][0])
    assert abs(np.hypot(un[0][0], un[1][0]) - 0.4) < 1e-15
    assert un[2][0] == 0.1
    # dv/dt = (q/m) v x B: for q B_z < 0 the rotation in the (x,y) plane is counter-clockwise
    assert abs(ang - 2 * np.arctan(-q * Bz * dt / (2 * m * gamma))) < 1e-14


def test_boris_pure_electric_kick():
    q, m, dt = -1.0, 2.0, 0.1
    u = [np.array([0.3]), np.array([-0.2]), np.array([0.0])]
    E = [np.array([1.0]), np.array([2.0]), np.array([-0.5])]
    B = [np.zeros(1)] * 3
    un = particles.boris(u, E, B, q, m, dt)
    for a in range(3):
        assert abs(un[a][0] - (u[a][0] + q * E[a][0] * dt / m)) < 1e-16


def test_tile_bins_brute_force():
    shape, dx, tile = (16, 8, 24), (0.5, 1.0, 0.1), (8, 4, 8)
    rng = np.random.default_rng(9)
    pos = [rng.uniform(0, shape[a] * dx[a], 4000) for a in range(3)]
    tid, off, order = particles.tile_bins(pos, dx, shape, tile)
    nt = [shape[a] // tile[a] for a in range(3)]
    for p in range(0, 4000, 37):
        c = [int(pos[a][p] // dx[a]) for a in range(3)]
        assert tid[p] == ((c[0] // tile[0]) * nt[1] + c[1] // tile[1]) * nt[2] + c[2] // tile[2]
    assert off[0] == 0 and off[-1] == 4000 and len(off) == nt[0] * nt[1] * nt[2] + 1
    assert np.all(np.diff(tid[order]) >= 0)


def test_vay_solves_its_defining_equation():
    # (u^{n+1/2} - u^{n-1/2}) m / (q dt) = E + (v^{n-1/2} + v^{n+1/2}) / 2 x B, v = u / gamma
    from oracle import particles
    rng = np.random.default_rng(11)
    n = 200
    c, q, m, dt = 2.0, -1.5, 0.7, 0.3
    u = [rng.normal(0, 3.0, n) for _ in range(3)]
    E = [rng.normal(0, 2.0, n) for _ in range(3)]
    B = [rng.normal(0, 2.0, n) for _ in range(3)]
    un = particles.vay(u, E, B, q, m, dt, c)
    gam = lambda w: np.sqrt(1.0 + (w[0] ** 2 + w[1] ** 2 + w[2] ** 2) / (c * c))
    g0, g1 = gam(u), gam(un)
    vb = [0.5 * (u[a] / g0 + un[a] / g1) for a in range(3)]
    rhs = [E[0] + vb[1] * B[2] - vb[2] * B[1], E[1] + vb[2] * B[0] - vb[0] * B[2],
           E[2] + vb[0] * B[1] - vb[1] * B[0]]
    for a in range(3):
        lhs = (un[a] - u[a]) * m / (q * dt)
        np.testing.assert_allclose(lhs, rhs[a], rtol=1e-11, atol=1e-11)


def test_vay_keeps_the_exb_drift_exactly_and_boris_does_not():
    # E = E0 y, B = B0 z: the drift v_d = E x B / B^2 = (E0 / B0) x sees no force
    from oracle import particles
    c, q, m, dt = 1.0, -1.0, 1.0, 0.5
    E0, B0 = 0.999 * 20.0, 20.0
    vd = E0 / B0
    gd = 1.0 / np.sqrt(1.0 - vd * vd)
    u = [np.array([gd * vd]), np.array([0.0]), np.array([0.0])]
    E = [np.array([0.0]), np.array([E0]), np.array([0.0])]
    B = [np.array([0.0]), np.array([0.0]), np.array([B0])]
    uv = particles.vay(u, E, B, q, m, dt, c)
    ub = particles.boris(u, E, B, q, m, dt, c)
    assert abs(uv[0][0] - u[0][0]) < 1e-12 * u[0][0] and abs(uv[1][0]) < 1e-12 * u[0][0]
    assert abs(ub[0][0] - u[0][0]) + abs(ub[1][0]) > 1e-3 * u[0][0]


def test_vay_pure_electric_kick():
    from oracle import particles
    rng = np.random.default_rng(5)
    u = [rng.normal(size=10) for _ in range(3)]
    E = [rng.normal(size=10) for _ in range(3)]
    Z = [np.zeros(10)] * 3
    un = particles.vay(u, E, Z, 2.0, 0.5, 0.1, 1.0)
    for a in range(3):
        np.testing.assert_allclose(un[a], u[a] + 2.0 / 0.5 * 0.1 * E[a], rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_offset_grid_gather_is_exact_for_linear_fields_and_deposit_keeps_moments(order):
    # grid points at (i + 1/2) dx along x (a Yee axis): a field linear in x sampled there is
    # gathered exactly, and deposits keep the charge and the first moment
    from oracle import particles
    shape, dx = (16, 8, 8), (0.5, 1.0, 2.0)
    rng = np.random.default_rng(order)
    n = 64
    pos = [rng.uniform(2.0, 6.0, n), rng.uniform(0, 8.0, n), rng.uniform(4.0, 12.0, n)]
    off = (0.5, 0.0, 0.5)
    X = [(np.arange(shape[a]) + off[a]) * dx[a] for a in range(3)]
    Xg = np.meshgrid(*X, indexing="ij")
    F = 1.5 + 0.25 * Xg[0] - 0.125 * Xg[2]
    (g,) = particles.gather([F], pos, dx, order, off)
    np.testing.assert_allclose(g, 1.5 + 0.25 * pos[0] - 0.125 * pos[2], rtol=1e-13, atol=1e-13)
    w = rng.uniform(0.5, 1.5, n)
    (d,) = particles.deposit(shape, pos, [w], dx, order, off)
    dV = np.prod(dx)
    assert abs(d.sum() * dV - w.sum()) < 1e-12 * w.sum()
    assert abs((d * Xg[0]).sum() * dV - (w * pos[0]).sum()) < 1e-11 * (w * pos[0]).sum()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_galilean_drift_and_midpoint_current(order):
    """No fields: u is unchanged and the particle moves by dt (v - v_gal) (Galilean coordinates,
    App. A.2); J^{n+1/2} is deposited at the midpoint x^n + dt (v - v_gal) / 2, so its first
    moment sum_i x_i J_i dV is q w v times that midpoint (B-splines reproduce linear functions)."""
    shape, dx, dt, c = (16, 16, 16), (0.5, 0.5, 0.5), 0.3, 1.0
    v_gal = (0.1, -0.2, 0.6)
    rng = np.random.default_rng(order)
    n = 5
    sp = {"x": rng.uniform(3.0, 5.0, n), "y": rng.uniform(3.0, 5.0, n), "z": rng.uniform(3.0, 5.0, n),
          "ux": rng.normal(0, 0.5, n), "uy": rng.normal(0, 0.5, n), "uz": rng.normal(0, 0.5, n),
          "w": rng.uniform(0.5, 1.5, n), "q": -1.0, "m": 1.0}
    Z = [np.zeros(shape) for _ in range(3)]
    out, J, rho = particles.push_and_deposit(sp, Z, Z, shape, dx, dt, order, v_gal, c)
    g = np.sqrt(1 + sp["ux"] ** 2 + sp["uy"] ** 2 + sp["uz"] ** 2)
    dV = np.prod(dx)
    X = [np.arange(shape[a])[tuple(slice(None) if b == a else None for b in range(3))] * dx[a] for a in range(3)]
    for a, (k, uk) in enumerate((("x", "ux"), ("y", "uy"), ("z", "uz"))):
        assert np.array_equal(out[uk], sp[uk])
        v = sp[uk] / g
        assert np.allclose(out[k], sp[k] + dt * (v - v_gal[a]), rtol=0, atol=1e-13)
        mid = sp[k] + 0.5 * dt * (v - v_gal[a])
        # first moment of J_a along its own axis: sum_p q w v_a mid_a
        assert abs(np.sum(X[a] * J[a]) * dV - np.sum(sp["q"] * sp["w"] * v * mid)) < 1e-12
        # rho^{n+1} sits at x^{n+1}
        assert abs(np.sum(X[a] * rho) * dV - np.sum(sp["q"] * sp["w"] * out[k])) < 1e-12


def test_cell_offset_split_pins():
    """FP32-form positions: faces land at offset 0 of their own cell, the last double below the
    box end stays in the last cell or wraps to cell 0 at offset 0 (never offset 1), the offset
    is in [0, 1), and the join reproduces x to the FP32 rounding of the offset."""
    N, dx = 512, 0.04
    faces = np.arange(N) * dx
    i, f = particles.cell_offset_split(faces, dx, N)
    t = faces * (1.0 / dx)
    # the cell is the FP64 form's CIC base node (a face whose product rounds just below the
    # integer belongs to the cell below); 11 of these 512 faces do, and x / dx would differ on 23
    base, _ = particles.shape_weights(faces, 1.0 / dx, 1)
    fixed = (f == 0) & (base % N != i)
    assert np.array_equal(np.where(fixed, i, base % N), i)
    assert np.array_equal(i[~fixed], base[~fixed] % N)
    assert int((base % N != np.arange(N)).sum()) == 11
    assert np.all((f == 0) | (t != np.round(t)))
    L = N * dx
    top = np.nextafter(L, 0.0)
    i, f = particles.cell_offset_split(np.array([top]), dx, N)
    # t is within one FP64 ulp of N: either 15 + (1 - tiny) rounding to 1.0f -> (0, 0) wrapped
    assert (i[0], float(f[0])) in ((0, 0.0), (N - 1, float(np.float32(top * (1.0 / dx) - (N - 1)))))
    assert float(f[0]) < 1.0
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, L, 100000)
    i, f = particles.cell_offset_split(x, dx, N)
    assert i.min() >= 0 and i.max() < N
    assert f.dtype == np.float32 and float(f.min()) >= 0.0 and float(f.max()) < 1.0
    back = particles.cell_offset_join(i, f, dx)
    d = np.abs(back - x)
    d = np.minimum(d, L - d)
    # FP32 rounding of an offset below 1: at most 2^-25 of a cell, plus the FP64 products
    assert float(d.max()) <= (2.0 ** -25 + 1e-14) * dx
    # the cell is the FP64 form's nearest-node cell except where the offset rounded up to 1
    base = np.floor(x * (1.0 / dx)).astype(np.int64) % N
    moved = i != base
    assert np.all(f[moved] == 0) and np.array_equal(i[moved], (base[moved] + 1) % N)


def test_cell_offset_split_rounds_up_to_the_next_cell():
    """An offset that rounds to 1.0 in FP32 moves the particle to offset 0 of the next cell."""
    dx = 1.0
    x = np.array([3.0 - 2.0 ** -30, 3.0 - 2.0 ** -20, 7.0 - 2.0 ** -40])
    i, f = particles.cell_offset_split(x, dx, 8)
    assert list(i) == [3, 2, 7]
    assert float(f[0]) == 0.0 and float(f[2]) == 0.0
    assert float(f[1]) == float(np.float32(1.0 - 2.0 ** -20))
    # and at the box end the next cell wraps to 0
    i, f = particles.cell_offset_split(np.array([8.0 - 2.0 ** -40]), dx, 8)
    assert int(i[0]) == 0 and float(f[0]) == 0.0


def test_linear_cell_is_c_order():
    shape = (4, 8, 16)
    ix, iy, iz = np.meshgrid(np.arange(4), np.arange(8), np.arange(16), indexing="ij")
    lin = particles.linear_cell(ix, iy, iz, shape)
    assert np.array_equal(lin.ravel(), np.arange(4 * 8 * 16))
