"""PSATD coefficients and k-space updates on the staggered (Yee) grid.

Test infrastructure only (see oracle/__init__.py).

Sec. 4.1 (notation), Sec. 4.2 (standard PSATD, Eqs. eq_update_B/E_with_rho_standard),
Sec. 4.3 (Galilean PSATD, Eqs. eq_update_B/E_with_rho_galilean),
Sec. 4.4 (averaged Galilean PSATD, Eqs. eq_update_B/E_with_rho_averaged).

Coefficients are evaluated per mode in long double from the paper's closed
forms, then rounded to complex128.  Where a closed form is 0/0 the limit is
taken explicitly:

* omega_s = 0 (only the k = 0 mode): the k -> 0 limits of S/omega_s, X1..X4,
  Psi1, Psi2, Psi3, Y1..Y4.
* Omega_c = 0 (v_gal . [k]_c = 0, e.g. the k_z = 0 plane): X2, X3 take their
  standard values (Sec. 4.3: the standard update is the Omega_c -> 0 limit),
  Psi3 -> 1, and Y2, Y3 take the Omega_c = 0 limits derived from the averaging
  that defines them (time average over [t^{n+1/2}, t^{n+3/2}] of the analytic
  solution, with rho linear in time):
      Y2 = -i (c^2/eps0) A1,  Y3 = -i (c^2/eps0) (A0 - A1),
      A0 = (1 - Psi1) / omega_s^2,
      A1 = (omega_s dt - (C1 - C3)/(omega_s dt)) / (omega_s^3 dt).
* X1 is written with chi_1 substituted (Eq. eq_chi1), so that omega_c^2 cancels:
      X1 = theta / (eps0 (omega_s^2 - Omega_c^2)) (theta* - theta C + i Omega_c theta S/omega_s).
"""
import numpy as np

from . import fornberg

LD = np.longdouble
CLD = np.clongdouble


def modified_wave_vectors(shape, dx, spectral_order):
    """Per-axis [k]_s and [k]_c (long double, 1D each) for the full (Nx, Ny, Nz) spectrum."""
    ks = [fornberg.k_staggered(shape[a], dx[a], spectral_order[a]) for a in range(3)]
    kc = [fornberg.k_centered(shape[a], dx[a], spectral_order[a]) for a in range(3)]
    return ks, kc


def _b3(v, a):
    s = [1, 1, 1]
    s[a] = v.shape[0]
    return v.reshape(s)


def coefficients(shape, dx, dt, spectral_order, v_gal=(0.0, 0.0, 0.0), c=1.0, eps0=1.0,
                 averaged=False, nodal=False):
    """Per-mode update coefficients, complex128 arrays of the full spectrum shape.

    Keys: 'TC' = theta_c^2 C, 'TS' = theta_c^2 S/omega_s, 'X1', 'X2', 'TX3' = theta_c^2 X3,
    'X4' (Secs. 4.2-4.3; theta_c = 1 when v_gal = 0) and, if averaged,
    'Psi1', 'Psi2', 'Y1', 'Y2', 'Y3', 'Y4' (Sec. 4.4).
    nodal: the nodal solver of the comparison cycle (Sec. 2), in which every quantity lives on
    the nodes and the centered modified wave numbers replace [k]_s (omega = c |[k]_c|).
    """
    ks, kc = modified_wave_vectors(shape, dx, spectral_order)
    if nodal:
        ks = kc = nodal_k(shape, kc, spectral_order)
    c = LD(c)
    eps0 = LD(eps0)
    dt = LD(dt)
    vg = [LD(v) for v in v_gal]
    ks2 = sum(_b3(ks[a], a) ** 2 for a in range(3))
    ws = c * np.sqrt(ks2)                                       # omega_s = c [k]_s
    Om = sum(vg[a] * _b3(kc[a], a) for a in range(3))           # Omega_c = v_gal . [k]_c
    ws, Om = np.broadcast_arrays(ws, Om)
    ws = ws.astype(LD)
    Om = Om.astype(LD)
    C = np.cos(ws * dt)
    S = np.sin(ws * dt)
    theta = np.exp(1j * Om * dt / 2).astype(CLD)
    thetas = np.conj(theta)
    z = ws == 0                       # only k = 0
    o = Om == 0
    wsn = np.where(z, LD(1), ws)      # safe denominators; limits patched below
    Omn = np.where(o, LD(1), Om)

    S_w = np.where(z, dt, S / wsn)                                        # S / omega_s
    one_m_C_w2 = np.where(z, dt * dt / 2, (1 - C) / wsn ** 2)            # (1 - C) / omega_s^2
    # standard coefficients (Sec. 4.2)
    X1s = one_m_C_w2 / eps0
    X2s = np.where(z, c * c * dt * dt / (6 * eps0),
                   c * c / (eps0 * wsn ** 2) * (1 - S / (wsn * dt)))
    X3s = np.where(z, -c * c * dt * dt / (3 * eps0),
                   c * c / (eps0 * wsn ** 2) * (C - S / (wsn * dt)))
    # Galilean coefficients (Sec. 4.3)
    den = ws * ws - Om * Om
    denn = np.where(z, LD(1), den)
    X1 = np.where(z, CLD(dt * dt / (2 * eps0)),
                  theta / (eps0 * denn) * (thetas - theta * C + 1j * Om * theta * S_w))
    dth = np.where(o, CLD(1), thetas - theta)
    X2 = np.where(o, X2s.astype(CLD), c * c / dth * (thetas * X1 - theta * one_m_C_w2 / eps0))
    X3 = np.where(o, X3s.astype(CLD), c * c / dth * (thetas * X1 - thetas * one_m_C_w2 / eps0))
    X4 = 1j * Om * X1 - theta ** 2 * S_w / eps0
    out = {
        "TC": theta ** 2 * C,
        "TS": theta ** 2 * S_w,
        "X1": X1, "X2": X2, "TX3": theta ** 2 * X3, "X4": X4,
    }
    if averaged:
        C1, S1 = np.cos(ws * dt / 2), np.sin(ws * dt / 2)
        C3, S3 = np.cos(3 * ws * dt / 2), np.sin(3 * ws * dt / 2)
        Psi1 = (theta ** 3 * (ws * S3 + 1j * Om * C3) - theta * (ws * S1 + 1j * Om * C1)) / (denn * dt)
        Psi2 = (theta ** 3 * (C3 - 1j * Om * S3 / wsn) - theta * (C1 - 1j * Om * S1 / wsn)) / (denn * dt)
        Psi1 = np.where(z, CLD(1), Psi1)
        Psi2 = np.where(z, CLD(-dt), Psi2)
        Psi3 = np.where(o, CLD(1), -1j * theta * (theta ** 2 - 1) / (Omn * dt))
        Y1 = np.where(z, CLD(13 * dt * dt / (24 * eps0)),
                      (1 - Psi1 - 1j * Om * Psi2) / (eps0 * denn))
        t2m1 = np.where(o, CLD(1), theta ** 2 - 1)
        Y2g = 1j * c * c * (eps0 * ws ** 2 * Y1 - Psi3 + Psi1) / (eps0 * wsn ** 2 * t2m1)
        Y3g = 1j * c * c * (Psi3 - Psi1 - eps0 * theta ** 2 * ws ** 2 * Y1) / (eps0 * wsn ** 2 * t2m1)
        A0 = np.where(z, 13 * dt * dt / 24, (1 - Psi1.real) / wsn ** 2)
        A1 = np.where(z, 5 * dt * dt / 24,
                      (wsn * dt - (C1 - C3) / (wsn * dt)) / (wsn ** 3 * dt))
        Y2 = np.where(o, -1j * c * c / eps0 * A1, Y2g)
        Y3 = np.where(o, -1j * c * c / eps0 * (A0 - A1), Y3g)
        Y4 = 1j * Om * Y1 + Psi2 / eps0
        out.update({"Psi1": Psi1, "Psi2": Psi2, "Y1": Y1, "Y2": Y2, "Y3": Y3, "Y4": Y4})
    return {k: np.asarray(v, dtype=CLD).astype(np.complex128) for k, v in out.items()}


def nodal_k(shape, kc, spectral_order):
    """[k]_c of the nodal solver: at infinite order its Nyquist entry (signed index -N/2) is
    set to 0, the centered derivative of a node-based field there (at finite order the sum of
    Eq. centered_modified_wave_number already gives 0); otherwise i [k]_c would break the
    Hermitian symmetry of real fields on the Nyquist planes."""
    out = []
    for a in range(3):
        k = kc[a].copy()
        if spectral_order[a] == 0 and shape[a] % 2 == 0:
            k[shape[a] // 2] = 0
        out.append(k)
    return out


def staggered_k_grid(shape, dx, spectral_order, nodal=False):
    """The three components of [k]_s (nodal: [k]_c, see nodal_k) broadcast to the spectrum
    shape, float64."""
    ks, kc = modified_wave_vectors(shape, dx, spectral_order)
    k = nodal_k(shape, kc, spectral_order) if nodal else ks
    return [np.broadcast_to(_b3(k[a].astype(np.float64), a), shape) for a in range(3)]


def cross(k, F):
    """k x F for 3-component lists."""
    return [k[1] * F[2] - k[2] * F[1], k[2] * F[0] - k[0] * F[2], k[0] * F[1] - k[1] * F[0]]


def update(Eh, Bh, Jh, rho_n, rho_np1, co, k, c=1.0):
    """One PSATD step in Fourier space (Galilean form; standard when theta_c = 1).

    Eq. eq_update_B_with_rho_galilean:
      B^{n+1} = theta^2 C B^n - i theta^2 (S/omega_s) [k]_s x E^n + i X1 [k]_s x J^{n+1/2}
    Eq. eq_update_E_with_rho_galilean:
      E^{n+1} = theta^2 C E^n + i c^2 theta^2 (S/omega_s) [k]_s x B^n + X4 J^{n+1/2}
                + i (theta^2 X3 rho^n - X2 rho^{n+1}) [k]_s
    (the standard Eqs. eq_update_B/E_with_rho_standard with theta = 1).
    """
    kxE = cross(k, Eh)
    kxB = cross(k, Bh)
    kxJ = cross(k, Jh)
    Bn = [co["TC"] * Bh[a] - 1j * co["TS"] * kxE[a] + 1j * co["X1"] * kxJ[a] for a in range(3)]
    En = [co["TC"] * Eh[a] + 1j * c * c * co["TS"] * kxB[a] + co["X4"] * Jh[a]
          + 1j * (co["TX3"] * rho_n - co["X2"] * rho_np1) * k[a] for a in range(3)]
    return En, Bn


def update_averaged(Eh, Bh, Jh, rho_n, rho_np1, co, k, c=1.0):
    """Averaged fields <E>^{n+1}, <B>^{n+1} (Eqs. eq_update_B/E_with_rho_averaged).

      <B> = Psi1 B^n + i Psi2 [k]_s x E^n + i Y1 [k]_s x J^{n+1/2}
      <E> = Psi1 E^n - i c^2 Psi2 [k]_s x B^n + Y4 J^{n+1/2} + (Y3 rho^n + Y2 rho^{n+1}) [k]_s
    """
    kxE = cross(k, Eh)
    kxB = cross(k, Bh)
    kxJ = cross(k, Jh)
    Ba = [co["Psi1"] * Bh[a] + 1j * co["Psi2"] * kxE[a] + 1j * co["Y1"] * kxJ[a] for a in range(3)]
    Ea = [co["Psi1"] * Eh[a] - 1j * c * c * co["Psi2"] * kxB[a] + co["Y4"] * Jh[a]
          + (co["Y3"] * rho_n + co["Y2"] * rho_np1) * k[a] for a in range(3)]
    return Ea, Ba
