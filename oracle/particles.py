"""Particle shapes, field gather, Boris push, direct deposition and tile bins.

Test infrastructure only (see oracle/__init__.py).

The paper fixes the shape family only as splines ("cubic splines", Sec. 5.2,
5.3); orders 1 and 2 come from the workloads.  These are the textbook
centred B-splines on the nodal grid, node i at i*dx:

  order 1: base = floor(t), d = t - base in [0,1); nodes base, base+1:
           (1-d, d)
  order 2: base = floor(t + 1/2), d = t - base in [-1/2,1/2); nodes base-1..base+1:
           ((1/2-d)^2/2, 3/4-d^2, (1/2+d)^2/2)
  order 3: base = floor(t), d = t - base in [0,1); nodes base-1..base+2:
           ((1-d)^3/6, (4-6d^2+3d^3)/6, (1+3d+3d^2-3d^3)/6, d^3/6)

with t = x * (1/dx) rounded to FP64 (the same single multiply on every side).

Boris push: the textbook scheme (half electric kick, magnetic rotation with
t = q B dt / (2 m gamma), s = 2 t / (1 + t^2), half electric kick); u is the
momentum per unit mass, u = gamma v.  In the Galilean variant the particle
moves by dt (v - v_gal) on the grid (Galilean coordinates x = x' - v_gal t,
App. A.2), while force and current use the lab velocity v.

Direct deposition (Sec. 2 cycle, deposit on the nodal grid; App. A.5 takes J
constant over the step): J^{n+1/2} = sum_p q w v^{n+1/2} S(x^{n+1/2} - x_i) / dV with
x^{n+1/2} = x^n + dt (v - v_gal) / 2, and rho^{n+1} = sum_p q w S(x^{n+1} - x_i) / dV.
"""
import numpy as np


def shape_weights(x, inv_dx, order, offset=0.0):
    """(lowest node index, weights[order+1, N]) of the order-`order` B-spline at positions x,
    for a grid whose node i sits at (i + offset) dx (offset 1/2: a staggered Yee axis)."""
    t = x * inv_dx - offset
    if order == 2:
        base = np.floor(t + 0.5)
    else:
        base = np.floor(t)
    d = t - base
    base = base.astype(np.int64)
    if order == 1:
        return base, np.stack([1.0 - d, d])
    if order == 2:
        return base - 1, np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2])
    if order == 3:
        return base - 1, np.stack([(1.0 - d) ** 3 / 6.0,
                                   (4.0 - 6.0 * d * d + 3.0 * d ** 3) / 6.0,
                                   (1.0 + 3.0 * d + 3.0 * d * d - 3.0 * d ** 3) / 6.0,
                                   d ** 3 / 6.0])
    raise ValueError("shape order must be 1, 2 or 3")


def _node_loop(pos, shape, dx, order, offset=(0.0, 0.0, 0.0)):
    """Yield (ix, iy, iz, S) for every one of the (order+1)^3 nodes around each particle
    (grid points at (i + offset_a) dx_a)."""
    lo, w = [], []
    for a in range(3):
        l, ww = shape_weights(pos[a], 1.0 / dx[a], order, offset[a])
        lo.append(l)
        w.append(ww)
    for i in range(order + 1):
        ix = (lo[0] + i) % shape[0]
        for j in range(order + 1):
            iy = (lo[1] + j) % shape[1]
            sxy = w[0][i] * w[1][j]
            for k in range(order + 1):
                iz = (lo[2] + k) % shape[2]
                yield ix, iy, iz, sxy * w[2][k]


def gather(fields, pos, dx, order, offset=(0.0, 0.0, 0.0)):
    """Interpolate fields (list of (Nx,Ny,Nz) arrays on the same grid, points at
    (i + offset) dx; nodal by default) to particle positions.

    F(x_p) = sum_{ijk} S(x_p - x_i) S(y_p - y_j) S(z_p - z_k) F_{ijk}  (gather step of Sec. 2).
    """
    shape = fields[0].shape
    out = [np.zeros_like(pos[0]) for _ in fields]
    for ix, iy, iz, S in _node_loop(pos, shape, dx, order, offset):
        for f, o in zip(fields, out):
            o += S * f[ix, iy, iz]
    return out


def deposit(grid_shape, pos, values, dx, order, offset=(0.0, 0.0, 0.0)):
    """Scatter per-particle values onto arrays with points at (i + offset) dx (nodal by
    default): rho_i = sum_p v_p S(x_p - x_i) / dV."""
    dV = dx[0] * dx[1] * dx[2]
    out = [np.zeros(grid_shape) for _ in values]
    for ix, iy, iz, S in _node_loop(pos, grid_shape, dx, order, offset):
        for v, o in zip(values, out):
            np.add.at(o, (ix, iy, iz), v * S)
    return [o / dV for o in out]


def boris(u, E, B, q, m, dt, c=1.0):
    """Textbook Boris rotation: u^{n-1/2} -> u^{n+1/2} with fields E, B at the particle."""
    k = q * dt / (2.0 * m)
    um = [u[a] + k * E[a] for a in range(3)]
    gm = np.sqrt(1.0 + (um[0] ** 2 + um[1] ** 2 + um[2] ** 2) / (c * c))
    t = [k * B[a] / gm for a in range(3)]
    s = [2.0 * t[a] / (1.0 + t[0] ** 2 + t[1] ** 2 + t[2] ** 2) for a in range(3)]
    up = [um[0] + (um[1] * t[2] - um[2] * t[1]),
          um[1] + (um[2] * t[0] - um[0] * t[2]),
          um[2] + (um[0] * t[1] - um[1] * t[0])]
    upl = [um[0] + (up[1] * s[2] - up[2] * s[1]),
           um[1] + (up[2] * s[0] - up[0] * s[2]),
           um[2] + (up[0] * s[1] - up[1] * s[0])]
    return [upl[a] + k * E[a] for a in range(3)]


def vay(u, E, B, q, m, dt, c=1.0):
    """Vay's pusher (J.-L. Vay, Phys. Plasmas 15, 056701 (2008); used for the paper's runs,
    Secs. 5.2-5.3): u^{n+1/2} - u^{n-1/2} = (q dt / m) (E + vbar x B) with vbar the mean of
    v^{n-1/2} and v^{n+1/2}, v = u / gamma, solved in closed form for u^{n+1/2}:
      u' = u + (q dt / m) (E + (v^{n-1/2} x B) / 2),   tau = (q dt / (2 m)) B,
      gamma^2 solves gamma^4 - sigma gamma^2 - (tau^2 + (u'.tau / c)^2) = 0,
      sigma = 1 + u'^2 / c^2 - tau^2,
      t = tau / gamma,  u^{n+1/2} = (u' + (u'.t) t + u' x t) / (1 + t^2).
    """
    g0 = np.sqrt(1.0 + (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / (c * c))
    v0 = [u[a] / g0 for a in range(3)]
    k = q * dt / m
    vxB = [v0[1] * B[2] - v0[2] * B[1], v0[2] * B[0] - v0[0] * B[2], v0[0] * B[1] - v0[1] * B[0]]
    up = [u[a] + k * (E[a] + 0.5 * vxB[a]) for a in range(3)]
    tau = [0.5 * k * B[a] for a in range(3)]
    tau2 = tau[0] ** 2 + tau[1] ** 2 + tau[2] ** 2
    ustar = (up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2]) / c
    sigma = 1.0 + (up[0] ** 2 + up[1] ** 2 + up[2] ** 2) / (c * c) - tau2
    gam = np.sqrt(0.5 * (sigma + np.sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))))
    t = [tau[a] / gam for a in range(3)]
    s = 1.0 / (1.0 + t[0] ** 2 + t[1] ** 2 + t[2] ** 2)
    ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2]
    uxt = [up[1] * t[2] - up[2] * t[1], up[2] * t[0] - up[0] * t[2], up[0] * t[1] - up[1] * t[0]]
    return [s * (up[a] + ut * t[a] + uxt[a]) for a in range(3)]


PUSHERS = {0: boris, 1: vay}


def wrap(x, L):
    """Periodic wrap of a position that moved by less than one box length."""
    x = np.where(x >= L, x - L, x)
    return np.where(x < 0.0, x + L, x)


# Yee offsets (in cells) of E, B and J components, for the staggered comparison cycle
_YEE_E = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))
_YEE_B = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))


def push_and_deposit(sp, nodal_E, nodal_B, grid_shape, dx, dt, order, v_gal=(0.0, 0.0, 0.0), c=1.0,
                     pusher=0, staggered=False):
    """Gather at x^n, push (Boris, or Vay with pusher = 1), move, and deposit J^{n+1/2} and
    rho^{n+1} for one species.

    sp: dict with x, y, z, ux, uy, uz, w (float64 arrays) and q, m (floats).
    staggered: the staggered comparison cycle of Sec. 2: E, B are gathered from their own Yee
    positions and J is deposited at its Yee positions (rho stays nodal).
    Returns (new species dict, [Jx, Jy, Jz] nodal (Yee if staggered), rho nodal).
    """
    L = [grid_shape[a] * dx[a] for a in range(3)]
    pos = [sp["x"], sp["y"], sp["z"]]
    if staggered:
        E = [gather([nodal_E[a]], pos, dx, order, _YEE_E[a])[0] for a in range(3)]
        B = [gather([nodal_B[a]], pos, dx, order, _YEE_B[a])[0] for a in range(3)]
    else:
        E = gather(nodal_E, pos, dx, order)
        B = gather(nodal_B, pos, dx, order)
    u = PUSHERS[pusher]([sp["ux"], sp["uy"], sp["uz"]], E, B, sp["q"], sp["m"], dt, c)
    g = np.sqrt(1.0 + (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / (c * c))
    v = [u[a] / g for a in range(3)]
    mid = [wrap(pos[a] + 0.5 * dt * (v[a] - v_gal[a]), L[a]) for a in range(3)]
    new = [wrap(pos[a] + dt * (v[a] - v_gal[a]), L[a]) for a in range(3)]
    qw = sp["q"] * sp["w"]
    if staggered:
        J = [deposit(grid_shape, mid, [qw * v[a]], dx, order, _YEE_E[a])[0] for a in range(3)]
    else:
        J = deposit(grid_shape, mid, [qw * v[0], qw * v[1], qw * v[2]], dx, order)
    (rho,) = deposit(grid_shape, new, [qw], dx, order)
    out = dict(sp)
    out.update(x=new[0], y=new[1], z=new[2], ux=u[0], uy=u[1], uz=u[2])
    return out, J, rho


def deposit_rho(sp, grid_shape, dx, order):
    """Charge density of one species at its current positions (rho^n for the first step)."""
    (rho,) = deposit(grid_shape, [sp["x"], sp["y"], sp["z"]], [sp["q"] * sp["w"]], dx, order)
    return rho


def tile_bins(pos, dx, grid_shape, tile):
    """Tile id of every particle and the per-tile offsets (exclusive prefix sum, length n_tiles+1).

    cell_a = floor(x_a * (1/dx_a)) mod N_a; tile_a = cell_a // tile_a;
    id = (tile_x * nty + tile_y) * ntz + tile_z.  Also returns a stable sort order.
    """
    nt = [grid_shape[a] // tile[a] for a in range(3)]
    cell = [np.floor(pos[a] * (1.0 / dx[a])).astype(np.int64) % grid_shape[a] for a in range(3)]
    tid = ((cell[0] // tile[0]) * nt[1] + cell[1] // tile[1]) * nt[2] + cell[2] // tile[2]
    counts = np.bincount(tid, minlength=nt[0] * nt[1] * nt[2])
    offsets = np.concatenate([[0], np.cumsum(counts)])
    order = np.argsort(tid, kind="stable")
    return tid, offsets, order


def cell_offset_split(x, dx, N):
    """Position of the FP32 form: integer cell index and FP32 offset inside that cell.

    The paper keeps positions in floating point; the FP32 form holds each coordinate as an
    integer cell i and an FP32 offset f in [0, 1) with x = (i + f) dx.  With t = x * (1/dx)
    rounded to FP64 (the single multiply of shape_weights, so the cell agrees with the FP64
    form's nearest-node rule), i = floor(t) and f = t - i (exact in FP64) rounded to FP32 once.
    When that rounding gives 1.0 the particle is put at offset 0 of the next cell.  The cell
    wraps periodically into [0, N).  Returns (i as int64, f as float32).
    """
    t = np.asarray(x, dtype=np.float64) * (1.0 / dx)
    base = np.floor(t)
    f = (t - base).astype(np.float32)
    up = f == np.float32(1.0)
    f = np.where(up, np.float32(0.0), f).astype(np.float32)
    i = (base.astype(np.int64) + up.astype(np.int64)) % N
    return i, f


def cell_offset_join(i, f, dx):
    """FP64 position x = (i + f) dx of a FP32-form coordinate (i + f is exact in FP64)."""
    return (np.asarray(i, dtype=np.int64).astype(np.float64) + np.asarray(f, dtype=np.float32).astype(np.float64)) * dx


def linear_cell(ix, iy, iz, shape):
    """Linear cell index (ix * Ny + iy) * Nz + iz of the C-order [Nx][Ny][Nz] grid."""
    return (np.asarray(ix, dtype=np.int64) * shape[1] + iy) * shape[2] + iz
