"""Diagnostics: electromagnetic field energy and the relative L2 error norm.

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
