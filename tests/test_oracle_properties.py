"""Property-based pins of the oracle (hypothesis draws the grids, spacings, orders and particles):
deposited charge equals the sum of q w, B-spline gathers reproduce linear fields exactly,
deposit and gather are adjoint, the two centering directions are transposes of each other, and
the FDTD curls satisfy div curl = 0 - for every drawn case, not just fixed seeds."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import fdtd, grid, particles  # noqa: E402

pow2 = st.sampled_from([4, 8, 16])
spacing = st.floats(min_value=0.1, max_value=2.0, allow_nan=False)
orders = st.integers(min_value=1, max_value=3)
SETTINGS = dict(max_examples=40, deadline=None)


def _case(seed, shape, dx, n):
    rng = np.random.default_rng(seed)
    L = [shape[a] * dx[a] for a in range(3)]
    pos = [rng.uniform(0, L[a], n) for a in range(3)]
    qw = rng.uniform(-2.0, 2.0, n)
    return rng, pos, qw


@settings(**SETTINGS)
@given(seed=st.integers(0, 2**31 - 1), nx=pow2, ny=pow2, nz=pow2, d=st.tuples(spacing, spacing, spacing),
       order=orders, n=st.integers(1, 200))
def test_charge_and_linear_gather(seed, nx, ny, nz, d, order, n):
    shape = (nx, ny, nz)
    rng, pos, qw = _case(seed, shape, d, n)
    (rho,) = particles.deposit(shape, pos, [qw], d, order)
    assert abs(rho.sum() * np.prod(d) - qw.sum()) < 1e-12 * max(1.0, np.abs(qw).sum())
    # a field linear along one axis (away from the periodic seam) is gathered exactly
    a = int(rng.integers(3))
    X = (np.arange(shape[a]) * d[a])
    f = np.broadcast_to(X[tuple(slice(None) if b == a else None for b in range(3))], shape).copy()
    L = shape[a] * d[a]
    inner = (pos[a] > 2.0 * d[a]) & (pos[a] < L - 3.0 * d[a])
    if inner.any():
        p_in = [q[inner] for q in pos]
        (g,) = particles.gather([f], p_in, d, order)
        assert np.max(np.abs(g - p_in[a])) < 1e-12 * L


@settings(**SETTINGS)
@given(seed=st.integers(0, 2**31 - 1), nx=pow2, ny=pow2, nz=pow2, d=st.tuples(spacing, spacing, spacing),
       order=orders, n=st.integers(1, 100))
def test_deposit_gather_adjoint(seed, nx, ny, nz, d, order, n):
    shape = (nx, ny, nz)
    rng, pos, qw = _case(seed, shape, d, n)
    F = rng.normal(size=shape)
    (dep,) = particles.deposit(shape, pos, [qw], d, order)
    (g,) = particles.gather([F], pos, d, order)
    lhs = np.sum(dep * F) * np.prod(d)
    rhs = np.sum(qw * g)
    assert abs(lhs - rhs) < 1e-11 * max(1.0, np.abs(qw).sum() * np.abs(F).max())


@settings(**SETTINGS)
@given(seed=st.integers(0, 2**31 - 1), n=st.sampled_from([8, 16, 32]), m=st.integers(1, 4),
       axis=st.integers(0, 2))
def test_centering_directions_are_transposes(seed, n, m, axis):
    rng = np.random.default_rng(seed)
    shape = [4, 4, 4]
    shape[axis] = n
    a = rng.normal(size=shape)
    b = rng.normal(size=shape)
    order = 2 * m
    lhs = np.sum(grid.center_staggered_to_nodal_1d(a, axis, order) * b)
    rhs = np.sum(a * grid.center_nodal_to_staggered_1d(b, axis, order))
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(a * a) * np.sum(b * b)) * n


@settings(**SETTINGS)
@given(seed=st.integers(0, 2**31 - 1), nx=pow2, ny=pow2, nz=st.sampled_from([8, 16, 32]),
       d=st.tuples(spacing, spacing, spacing), o=st.tuples(*(st.sampled_from([2, 4, 6, 8]),) * 3))
def test_fdtd_div_curl_vanishes(seed, nx, ny, nz, d, o):
    shape = (nx, ny, nz)
    orders = tuple(min(k, s) for k, s in zip(o, shape))
    rng = np.random.default_rng(seed)
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    scale = (1.0 / min(d)) ** 2 * 10
    assert np.max(np.abs(fdtd.div_B(fdtd.curl_E(E, orders, d), orders, d))) < 1e-12 * scale
    assert np.max(np.abs(fdtd.div_E(fdtd.curl_B(B, orders, d), orders, d))) < 1e-12 * scale
