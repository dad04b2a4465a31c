"""Seeded synthetic inputs for the hybrid PSATD PIC step.

This module only draws random numbers and evaluates the initial conditions of
the benchmark workloads; it holds none of the method's arithmetic and is shared
by the tests, the benchmark and the CPU reference.  Every workload mirrors one
of the paper's test problems in shape, parameter range and structure (a
thermal plasma, the laser-wakefield box of Sec. 5.2, a drifting pair plasma
for the Galilean solver, a differentiable probe problem, the beam-driven
wakefield box of Sec. 5.3); none reads a dataset.

Units: normalised plasma units, c = eps0 = mu0 = 1, electron q = -1, m = 1,
density n0 = 1.  Weights are w = n(x) dV / ppc.  Fields on the Yee grid (each
component at its own position; rho nodal), arrays (Nx, Ny, Nz) float64.
"""
import numpy as np

STANDARD, GALILEAN, AVERAGED = 0, 1, 2

# Yee positions of each field component, in units of the cell size (layout contract).
_YEE_OFFSET = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
}


def _coords(shape, dx, name):
    off = _YEE_OFFSET[name]
    ax = [(np.arange(shape[a]) + off[a]) * dx[a] for a in range(3)]
    return np.meshgrid(*ax, indexing="ij")


def _stratified(rng, shape, dx, ppc, density=None):
    """ppc particles uniformly placed in every cell; weight w = n dV / ppc."""
    n_cells = shape[0] * shape[1] * shape[2]
    idx = np.repeat(np.arange(n_cells, dtype=np.int64), ppc)
    ix, rem = np.divmod(idx, shape[1] * shape[2])
    iy, iz = np.divmod(rem, shape[2])
    u = rng.random((3, idx.size))
    x = (ix + u[0]) * dx[0]
    y = (iy + u[1]) * dx[1]
    z = (iz + u[2]) * dx[2]
    dV = dx[0] * dx[1] * dx[2]
    n = np.ones(idx.size) if density is None else density(x, y, z)
    w = n * dV / ppc
    return x, y, z, w


def _species(x, y, z, ux, uy, uz, w, q, m):
    return {"x": x, "y": y, "z": z, "ux": ux, "uy": uy, "uz": uz, "w": w, "q": float(q), "m": float(m)}


def _zeros(shape):
    return [np.zeros(shape) for _ in range(3)]


def thermal_plasma(shape=(32, 32, 32), ppc=8, seed=1001, u_th=0.01, steps=10):
    """Thermal electron plasma, 32^3, dx = 1, dt = dz/c, standard PSATD (infinite order),
    centering order 8, CIC, 8 particles per cell, E = B = 0, 10 steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = (1.0, 1.0, 1.0)
    x, y, z, w = _stratified(rng, shape, dx, ppc)
    u = rng.normal(0.0, u_th, (3, x.size))
    return {
        "name": "thermal_plasma_%dx%dx%d" % shape,
        "params": dict(shape=shape, dx=dx, dt=1.0, shape_order=1, centering_order=(8, 8, 8),
                       variant=STANDARD, v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0),
        "E": _zeros(shape), "B": _zeros(shape),
        "species": [_species(x, y, z, u[0], u[1], u[2], w, -1.0, 1.0)],
        "steps": steps,
    }


def laser_wakefield(shape=(128, 128, 512), ppc=2, seed=1002, steps=200, a0=2.0):
    """Laser-wakefield box: dx = dy = 0.2, dz = 0.04, dt = dz/c, standard PSATD (infinite
    order), centering (8, 8, 16), cubic shape, cold electrons with a 50-cell linear up-ramp,
    2 per cell, and a Gaussian laser (a0 = 2, 30 cells per wavelength along z, waist 20 cells,
    duration 60 cells, centred 150 cells into the box) polarised along y, moving along +z."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = (0.2, 0.2, 0.04)
    ramp = 50 * dx[2]
    x, y, z, w = _stratified(rng, shape, dx, ppc, density=lambda x, y, z: np.minimum(1.0, z / ramp))
    zeros = np.zeros_like(x)
    k0 = 2 * np.pi / (30 * dx[2])
    E0 = a0 * k0                        # a0 * omega0 with c = 1
    w0 = 20 * dx[0]
    L = 60 * dx[2]
    zL = 150 * dx[2]
    xc = shape[0] * dx[0] / 2
    yc = shape[1] * dx[1] / 2

    def profile(X, Y, Z):
        r2 = (X - xc) ** 2 + (Y - yc) ** 2
        return E0 * np.exp(-r2 / w0 ** 2) * np.exp(-((Z - zL) / L) ** 2) * np.cos(k0 * (Z - zL))

    E = _zeros(shape)
    B = _zeros(shape)
    E[1] = profile(*_coords(shape, dx, "Ey"))
    B[0] = -profile(*_coords(shape, dx, "Bx"))
    return {
        "name": "laser_wakefield_%dx%dx%d" % shape,
        "params": dict(shape=shape, dx=dx, dt=dx[2], shape_order=3, centering_order=(8, 8, 16),
                       variant=STANDARD, v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0),
        "E": E, "B": B,
        "species": [_species(x, y, z, zeros, zeros.copy(), zeros.copy(), w, -1.0, 1.0)],
        "steps": steps,
    }


def galilean_drift(shape=(64, 64, 256), ppc=2, seed=1003, gamma=130.0, u_th=1e-3, steps=500):
    """Drifting electron-positron plasma for the Galilean solver: dx = 1, dt = dz/c,
    v_gal = plasma drift (gamma = 130 along z), spectral order 16, centering order 8,
    quadratic shape, 2 electrons + 2 positrons per cell (co-located, independent momenta)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = (1.0, 1.0, 1.0)
    beta = np.sqrt(1.0 - 1.0 / gamma ** 2)
    x, y, z, w = _stratified(rng, shape, dx, ppc)
    ue = rng.normal(0.0, u_th, (3, x.size))
    up = rng.normal(0.0, u_th, (3, x.size))
    ue[2] += gamma * beta
    up[2] += gamma * beta
    sp = [_species(x, y, z, ue[0], ue[1], ue[2], w, -1.0, 1.0),
          _species(x.copy(), y.copy(), z.copy(), up[0], up[1], up[2], w.copy(), 1.0, 1.0)]
    return {
        "name": "galilean_drift_%dx%dx%d" % shape,
        "params": dict(shape=shape, dx=dx, dt=1.0, shape_order=2, centering_order=(8, 8, 8),
                       variant=GALILEAN, v_gal=(0.0, 0.0, beta), spectral_order=(16, 16, 16),
                       c=1.0, eps0=1.0),
        "E": _zeros(shape), "B": _zeros(shape),
        "species": sp, "steps": steps,
    }


def seed_wave(shape=(64, 64, 64), ppc=4, seed=1004, amplitude=1e-2, u_th=0.05, steps=50):
    """Differentiable probe problem: 64^3, dx = 1, dt = dz/c, standard PSATD, CIC, centering 8,
    4 electrons per cell with u_th = 0.05 and a Gaussian seed wave of amplitude A in E_x:
    E_x = A exp(-((z - Nz/2)/8)^2) cos(2 pi z / 16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = (1.0, 1.0, 1.0)
    x, y, z, w = _stratified(rng, shape, dx, ppc)
    u = rng.normal(0.0, u_th, (3, x.size))
    E = _zeros(shape)
    Z = _coords(shape, dx, "Ex")[2]
    zc = shape[2] * dx[2] / 2
    E[0] = amplitude * np.exp(-((Z - zc) / 8.0) ** 2) * np.cos(2 * np.pi * Z / 16.0)
    return {
        "name": "seed_wave_%dx%dx%d" % shape,
        "params": dict(shape=shape, dx=dx, dt=1.0, shape_order=1, centering_order=(8, 8, 8),
                       variant=STANDARD, v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0),
        "E": E, "B": _zeros(shape),
        "species": [_species(x, y, z, u[0], u[1], u[2], w, -1.0, 1.0)],
        "steps": steps,
        "probe": (tuple(s // 2 - 8 for s in shape), tuple(s // 2 + 8 for s in shape)),
    }


def beam_wakefield(shape=(256, 256, 1024), ppc=1, n_beam=1_000_000, seed=1005, gamma_b=1000.0,
                   steps=100):
    """Beam-driven wakefield box: dx = dy = 0.1, dz = 0.02, dt = dz/c, averaged Galilean PSATD
    with v_gal = beam velocity, spectral order 16, centering (8, 8, 16), cubic shape; cold
    plasma at 1 per cell plus a Gaussian electron driver (sigma_r = 4 cells, sigma_z = 10
    cells, gamma = 1000, peak density 10 n0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = (0.1, 0.1, 0.02)
    beta = np.sqrt(1.0 - 1.0 / gamma_b ** 2)
    x, y, z, w = _stratified(rng, shape, dx, ppc)
    zeros = np.zeros_like(x)
    sr, sz = 4 * dx[0], 10 * dx[2]
    L = [shape[a] * dx[a] for a in range(3)]
    c0 = (L[0] / 2, L[1] / 2, 0.75 * L[2])
    g = rng.normal(0.0, 1.0, (3, n_beam))
    bx = np.mod(c0[0] + sr * g[0], L[0])
    by = np.mod(c0[1] + sr * g[1], L[1])
    bz = np.mod(c0[2] + sz * g[2], L[2])
    wb = np.full(n_beam, 10.0 * (2 * np.pi) ** 1.5 * sr * sr * sz / n_beam)
    bzeros = np.zeros(n_beam)
    uz = np.full(n_beam, np.sqrt(gamma_b ** 2 - 1.0))
    sp = [_species(x, y, z, zeros, zeros.copy(), zeros.copy(), w, -1.0, 1.0),
          _species(bx, by, bz, bzeros, bzeros.copy(), uz, wb, -1.0, 1.0)]
    return {
        "name": "beam_wakefield_%dx%dx%d" % shape,
        "params": dict(shape=shape, dx=dx, dt=dx[2], shape_order=3, centering_order=(8, 8, 16),
                       variant=AVERAGED, v_gal=(0.0, 0.0, beta), spectral_order=(16, 16, 16),
                       c=1.0, eps0=1.0),
        "E": _zeros(shape), "B": _zeros(shape),
        "species": sp, "steps": steps,
    }


WORKLOADS = {
    "thermal_plasma": thermal_plasma,
    "laser_wakefield": laser_wakefield,
    "galilean_drift": galilean_drift,
    "seed_wave": seed_wave,
    "beam_wakefield": beam_wakefield,
}
