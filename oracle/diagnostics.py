"""Diagnostics: field energy, relative L2 error norm, stencil extent, beam RMS,
numerical vacuum dispersion.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np


def field_energy(E, B, dx, c=1.0, eps0=1.0, box_lo=None, box_hi=None):
    """W = 1/2 sum_cells (eps0 |E|^2 + |B|^2 / mu0) dV (Sec. 2, item (iii)), mu0 = 1/(eps0 c^2).

    Each Yee component is summed over its own array elements with index in
    [box_lo, box_hi) per axis (whole grid by default).
    """
    mu0 = 1.0 / (eps0 * c * c)
    dV = dx[0] * dx[1] * dx[2]
    shape = E[0].shape
    lo = box_lo or (0, 0, 0)
    hi = box_hi or shape
    sl = tuple(slice(lo[a], hi[a]) for a in range(3))
    we = sum(float(np.sum(E[a][sl] ** 2)) for a in range(3))
    wb = sum(float(np.sum(B[a][sl] ** 2)) for a in range(3))
    return 0.5 * (eps0 * we + wb / mu0) * dV


def l2_relative_error(a, b):
    """||a - b||_2 / ||b||_2 (Sec. 5.2, Eq. L2_norm_error); 0 when both vanish."""
    nb = float(np.linalg.norm(np.ravel(b)))
    na = float(np.linalg.norm(np.ravel(a) - np.ravel(b)))
    if nb == 0.0:
        return na
    return na / nb


def stencil_extent(g, axis):
    """Stencil extent of a Fourier-space quantity g along one axis (Sec. 2 (ii),
    Eq. stencil_extent): the inverse DFT of g along `axis`, averaged over the Fourier
    indices of the two other axes, in modulus.  g is given on the full spectrum
    (numpy FFT order); returns Gamma(x_j), j = 0 .. N_axis - 1 (x_j = j dx, periodic).
    """
    h = np.fft.ifft(np.asarray(g, dtype=np.complex128), axis=axis)
    others = tuple(a for a in range(3) if a != axis)
    return np.abs(np.mean(h, axis=others))


def beam_rms(x, y, w):
    """Averaged transverse RMS size of a particle beam (Sec. 5.3, Eq. RMS_pwfa):
    delta = 1/2 sqrt(sum w (x - <x>)^2 / sum w) + 1/2 sqrt(sum w (y - <y>)^2 / sum w),
    <.> the w-weighted means."""
    x, y, w = (np.asarray(a, dtype=np.float64) for a in (x, y, w))
    sw = np.sum(w)
    mx, my = np.sum(w * x) / sw, np.sum(w * y) / sw
    return 0.5 * np.sqrt(np.sum(w * (x - mx) ** 2) / sw) + 0.5 * np.sqrt(np.sum(w * (y - my) ** 2) / sw)


def vacuum_dispersion(co, k, axis, c=1.0, dt=1.0):
    """Numerical vacuum frequency of a PSATD update for waves along `axis` (Sec. 2 (i),
    App. B): for every Fourier index m along the axis (the other indices 0), the update of
    `update` (oracle/psatd.py) restricted to one transverse polarisation (E along the next
    axis, B along the one after) is applied to unit inputs, giving a 2x2 matrix per mode;
    omega = (largest phase of its two eigenvalues) / dt.

    co: full-spectrum coefficient tables (oracle/psatd.coefficients), k: the three [k]_s
    components broadcast to the spectrum shape.  Returns omega for m = 0 .. N_axis - 1
    (numpy FFT order)."""
    from . import psatd
    shape = co["TC"].shape
    n = shape[axis]
    e_ax, b_ax = (axis + 1) % 3, (axis + 2) % 3
    out = np.zeros(n)
    for m in range(n):
        idx = [0, 0, 0]
        idx[axis] = m
        idx = tuple(idx)
        M = np.zeros((2, 2), dtype=np.complex128)
        for col, (fe, fb) in enumerate(((1.0, 0.0), (0.0, 1.0))):
            E = [np.zeros(shape, dtype=np.complex128) for _ in range(3)]
            B = [np.zeros(shape, dtype=np.complex128) for _ in range(3)]
            E[e_ax][idx] = fe
            B[b_ax][idx] = fb
            zero = [np.zeros(shape, dtype=np.complex128) for _ in range(3)]
            rz = np.zeros(shape, dtype=np.complex128)
            En, Bn = psatd.update(E, B, zero, rz, rz, co, k, c)
            M[0, col] = En[e_ax][idx]
            M[1, col] = Bn[b_ax][idx]
        out[m] = np.max(np.angle(np.linalg.eigvals(M))) / dt
    return out
