"""Yee staggering, discrete Fourier conventions and finite-order centering.

Test infrastructure only (see oracle/__init__.py).

Real-space arrays have shape (Nx, Ny, Nz), C order (z fastest).  Node (i,j,k)
sits at (i dx, j dy, k dz); a component staggered along an axis sits half a
cell further along that axis (App. A, the list of Yee positions):

    E^x, J^x: (i+1/2, j, k)      B^x: (i, j+1/2, k+1/2)
    E^y, J^y: (i, j+1/2, k)      B^y: (i+1/2, j, k+1/2)
    E^z, J^z: (i, j, k+1/2)      B^z: (i+1/2, j+1/2, k)
    rho: nodal (i, j, k)

The staggering vector s in {0,1}^3 of each component is STAG[name].

Fourier convention (App. A.1, Eqs. Fourier_discrete and
Fourier_discrete_staggered): f_hat(k) = sum_j f_j exp(-i k . x_j) with x_j the
component's own position, i.e. the plain DFT times exp(-i k_a dx_a / 2) along
every staggered axis a.  k_a takes the signed values of fornberg.wave_numbers
(Nyquist at -pi/dx).
"""
import numpy as np

from . import fornberg

STAG = {
    "Ex": (1, 0, 0), "Ey": (0, 1, 0), "Ez": (0, 0, 1),
    "Bx": (0, 1, 1), "By": (1, 0, 1), "Bz": (1, 1, 0),
    "Jx": (1, 0, 0), "Jy": (0, 1, 0), "Jz": (0, 0, 1),
    "rho": (0, 0, 0),
}
E_NAMES = ("Ex", "Ey", "Ez")
B_NAMES = ("Bx", "By", "Bz")
J_NAMES = ("Jx", "Jy", "Jz")


# ---------------------------------------------------------------------------
# Finite-order centering (Sec. 3, Eq. staggered_finite_sum)
# ---------------------------------------------------------------------------

def center_staggered_to_nodal_1d(f, axis, order):
    """Interpolate a quantity staggered along `axis` onto the nodes of that axis.

    Eq. staggered_finite_sum: f_j = sum_{n=1}^{m} alpha^s_{m,n} (f_{j+n-1/2} + f_{j-n+1/2}) / 2,
    2m = order, periodic.  Array element s[i] holds the value at (i + 1/2) dx,
    so f_{j+n-1/2} = s[j+n-1] and f_{j-n+1/2} = s[j-n].
    """
    out = np.zeros_like(f)
    for n, a in enumerate(fornberg.alpha_staggered(order // 2), start=1):
        w = float(a) / 2.0
        out += w * (np.roll(f, -(n - 1), axis=axis) + np.roll(f, n, axis=axis))
    return out


def center_nodal_to_staggered_1d(f, axis, order):
    """Interpolate a nodal quantity onto the cell centers of `axis`.

    The paper states the centering only in the staggered -> nodal direction
    (Eq. staggered_finite_sum); the nodal -> staggered direction is its mirror
    image:  f_{j+1/2} = sum_n alpha^s_{m,n} (f_{j+n} + f_{j-n+1}) / 2, periodic.
    Output element s[j] holds the value at (j + 1/2) dx.
    """
    out = np.zeros_like(f)
    for n, a in enumerate(fornberg.alpha_staggered(order // 2), start=1):
        w = float(a) / 2.0
        out += w * (np.roll(f, -n, axis=axis) + np.roll(f, n - 1, axis=axis))
    return out


def center_to_nodal(f, name, orders):
    """Center a Yee component onto the nodal grid, one staggered axis at a time (x, y, z order)."""
    for a, s in enumerate(STAG[name]):
        if s:
            f = center_staggered_to_nodal_1d(f, a, orders[a])
    return f


def center_to_yee(f, name, orders):
    """Center a nodal array onto the Yee position of component `name` (x, y, z order)."""
    for a, s in enumerate(STAG[name]):
        if s:
            f = center_nodal_to_staggered_1d(f, a, orders[a])
    return f


# ---------------------------------------------------------------------------
# Discrete Fourier conventions (App. A.1)
# ---------------------------------------------------------------------------

def shift_factor(shape, dx, stag, sign):
    """prod_a exp(sign * i k_a dx_a / 2) over the staggered axes of `stag`, as complex128.

    k_a dx_a / 2 = pi j / N_a for signed index j: evaluated with exact reduction.
    """
    out = np.ones(shape, dtype=np.complex128)
    for a, s in enumerate(stag):
        if not s:
            continue
        N = shape[a]
        j = fornberg.signed_index(N)
        c = fornberg.cos_pi_frac(j, N).astype(np.float64)
        sn = fornberg.sin_pi_frac(j, N).astype(np.float64)
        f1 = c + 1j * sign * sn
        bshape = [1, 1, 1]
        bshape[a] = N
        out = out * f1.reshape(bshape)
    return out


def to_spectral(f, name, dx):
    """Paper-convention spectrum of a real-space component (Eqs. Fourier_discrete(_staggered))."""
    return np.fft.fftn(f) * shift_factor(f.shape, dx, STAG[name], -1)


def from_spectral(fh, name, dx):
    """Inverse of to_spectral.  Returns (real part, max |imaginary part|)."""
    g = np.fft.ifftn(fh * shift_factor(fh.shape, dx, STAG[name], +1))
    return g.real.copy(), float(np.max(np.abs(g.imag))) if g.size else 0.0


def positions(shape, dx, name):
    """Physical coordinates (X, Y, Z) of every element of component `name` (App. A)."""
    ax = [(np.arange(shape[a]) + 0.5 * STAG[name][a]) * dx[a] for a in range(3)]
    return np.meshgrid(*ax, indexing="ij")


def bilinear_filter(f, passes):
    """`passes` passes of the bilinear (1/4, 1/2, 1/4) smoothing filter along every axis
    of a periodic array (Sec. 2: the optional smoothing of the deposited rho and J,
    Birdsall and Langdon): f_j <- f_{j-1}/4 + f_j/2 + f_{j+1}/4, axes x, y, z in turn."""
    g = np.asarray(f, dtype=np.float64)
    for _ in range(int(passes)):
        for a in range(g.ndim):
            g = 0.25 * np.roll(g, 1, axis=a) + 0.5 * g + 0.25 * np.roll(g, -1, axis=a)
    return g
