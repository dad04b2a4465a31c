"""Finite-difference (FDTD) Maxwell solver on the Yee grid, for the hybrid FDTD cycle.

Test infrastructure only (see oracle/__init__.py).

The conclusions (Sec. 6) note that the hybrid scheme carries over to FDTD solvers: the fields
are advanced on the Yee grid by finite differences instead of the PSATD update, and the
finite-order centering of Sec. 3 still moves E, B to the nodes for the gather and the nodal J
to the Yee grid.  This module is that solver, written from its textbook definition:

* Staggered derivative of order 2m along an axis (the real-space form of [k]_s, Eq.
  staggered_modified_wave_number): a quantity sampled on the nodes of that axis is
  differentiated onto the half-integer points and vice versa,

      (D f)_{j+1/2} = sum_{n=1}^{m} c_n (f_{j+n} - f_{j-n+1}) / dx,
      c_n = alpha^s_{m,n} / (2n - 1),

  whose symbol on exp(i k x) is i [k]_s.  m = 1 is Yee's difference (c_1 = 1); m = 2 gives
  the textbook (9/8, -1/24).
* Curls: curl E lands on the B positions (E is nodal along the axes it is differentiated
  along), curl B on the E positions (B is staggered along them).
* Time stepping: leapfrog with the B update split in two halves so that E and B are both
  known at integer times (the state of the PIC cycle):
      B^{n+1/2} = B^n - (dt/2) curl E^n
      E^{n+1}   = E^n + dt (c^2 curl B^{n+1/2} - J^{n+1/2} / eps0)
      B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}
  (Maxwell's equations as in Sec. 4: dB/dt = -curl E, dE/dt = c^2 curl B - J / eps0.)
"""
import numpy as np

from . import fornberg


def fd_weights(order, dx):
    """c_n / dx for n = 1..m, 2m = order (FP64)."""
    m = int(order) // 2
    return [float(a / (2 * n - 1)) / dx for n, a in enumerate(fornberg.alpha_staggered(m), start=1)]


def d_to_half(f, axis, order, dx):
    """Derivative along `axis` of a quantity on the nodes of that axis, at the half points.

    Output element j holds the value at (j + 1/2) dx: sum_n c_n (f[j+n] - f[j-n+1]) / dx.
    """
    out = np.zeros_like(f)
    for n, w in enumerate(fd_weights(order, dx), start=1):
        out += w * (np.roll(f, -n, axis=axis) - np.roll(f, n - 1, axis=axis))
    return out


def d_to_node(s, axis, order, dx):
    """Derivative along `axis` of a quantity on the half points of that axis, at the nodes.

    s[i] holds the value at (i + 1/2) dx; output j: sum_n c_n (s[j+n-1] - s[j-n]) / dx.
    """
    out = np.zeros_like(s)
    for n, w in enumerate(fd_weights(order, dx), start=1):
        out += w * (np.roll(s, -(n - 1), axis=axis) - np.roll(s, n, axis=axis))
    return out


def curl_E(E, orders, dx):
    """curl E at the B positions: (d_y E^z - d_z E^y, d_z E^x - d_x E^z, d_x E^y - d_y E^x)."""
    Ex, Ey, Ez = E
    D = lambda f, a: d_to_half(f, a, orders[a], dx[a])
    return [D(Ez, 1) - D(Ey, 2), D(Ex, 2) - D(Ez, 0), D(Ey, 0) - D(Ex, 1)]


def curl_B(B, orders, dx):
    """curl B at the E positions (B is staggered along the axes it is differentiated along)."""
    Bx, By, Bz = B
    D = lambda f, a: d_to_node(f, a, orders[a], dx[a])
    return [D(Bz, 1) - D(By, 2), D(Bx, 2) - D(Bz, 0), D(By, 0) - D(Bx, 1)]


def div_E(E, orders, dx):
    """Divergence of a Yee E (or J) at the nodes."""
    return sum(d_to_node(E[a], a, orders[a], dx[a]) for a in range(3))


def div_B(B, orders, dx):
    """Divergence of a Yee B at the cell centers (i + 1/2, j + 1/2, k + 1/2)."""
    return sum(d_to_half(B[a], a, orders[a], dx[a]) for a in range(3))


def yee_update(E, B, J, dt, orders, dx, c=1.0, eps0=1.0):
    """One leapfrog step with split B: (E^n, B^n, J^{n+1/2}) -> (E^{n+1}, B^{n+1}), Yee grid."""
    h = 0.5 * dt
    cE = curl_E(E, orders, dx)
    Bh = [B[a] - h * cE[a] for a in range(3)]
    cB = curl_B(Bh, orders, dx)
    En = [E[a] + dt * (c * c * cB[a] - J[a] / eps0) for a in range(3)]
    cE = curl_E(En, orders, dx)
    Bn = [Bh[a] - h * cE[a] for a in range(3)]
    return En, Bn


def courant_limit(orders, dx, c=1.0):
    """Largest stable dt: c dt sqrt(sum_a max_k [k_a]_s^2) <= 2, the maximum at the Nyquist
    wave number, where [k]_s = (2 / dx) sum_n c_n (-1)^(n+1)."""
    s = 0.0
    for a in range(3):
        kmax = 2.0 * sum(w * (1 if n % 2 else -1) for n, w in enumerate(fd_weights(orders[a], dx[a]), start=1))
        s += kmax * kmax
    return 2.0 / (c * np.sqrt(s))
