"""Invariants of the full hybrid cycle (oracle.step): there is no closed form for a
multi-step PIC run, so the full step is pinned compositionally (every stage has
its own pins) plus these invariants: total charge, vacuum energy, and the
cold-plasma (Langmuir) oscillation at omega_p."""
import numpy as np
import pytest

from oracle import diagnostics, grid, psatd, step
from paper_2106_12919_gb300 import workloads


def _state(w):
    p = step.Params(**w["params"])
    st = {"E": [a.copy() for a in w["E"]], "B": [a.copy() for a in w["B"]],
          "species": [dict(s) for s in w["species"]]}
    st["rho"] = step.initial_rho(p, st["species"])
    return p, st


@pytest.mark.parametrize("name,kw", [
    ("thermal_plasma", dict(shape=(8, 8, 8), ppc=2)),
    ("laser_wakefield", dict(shape=(8, 8, 32), ppc=1)),
    ("galilean_drift", dict(shape=(8, 8, 16), ppc=1)),
    ("beam_wakefield", dict(shape=(8, 8, 32), ppc=1, n_beam=200)),
])
def test_charge_conserved_and_real(name, kw):
    w = workloads.WORKLOADS[name](**kw)
    p, st = _state(w)
    qtot = sum(float(np.sum(s["q"] * s["w"])) for s in st["species"])
    qabs = sum(float(np.sum(np.abs(s["q"] * s["w"]))) for s in st["species"])
    dV = np.prod(p.dx)
    for _ in range(3):
        step.hybrid_step(p, st)
        assert abs(np.sum(st["rho"]) * dV - qtot) < 1e-12 * qabs
        assert st["max_imag"] < 1e-9 * max(1.0, max(np.abs(e).max() for e in st["E"]))
        for a in range(3):
            assert np.all(np.isfinite(st["E"][a])) and np.all(np.isfinite(st["B"][a]))


@pytest.mark.parametrize("variant,order,v", [(0, (0, 0, 0), 0.0), (1, (16, 16, 16), 0.9),
                                             (2, (8, 8, 8), 0.5)])
def test_vacuum_energy_conserved(variant, order, v):
    shape, dx, dt = (8, 8, 16), (1.0, 0.8, 0.5), 0.45
    p = step.Params(shape, dx, dt, 1, (8, 8, 8), variant, (0.0, 0.0, v), order)
    rng = np.random.default_rng(1)
    k = psatd.staggered_k_grid(shape, dx, order)
    k2 = sum(k[a] ** 2 for a in range(3))
    k2s = np.where(k2 == 0, 1.0, k2)

    def solenoidal(names):
        F = [grid.to_spectral(rng.normal(size=shape), n, dx) for n in names]
        kd = sum(k[a] * F[a] for a in range(3)) / k2s
        return [grid.from_spectral(F[a] - k[a] * kd, names[a], dx)[0] for a in range(3)]

    st = {"E": solenoidal(grid.E_NAMES), "B": solenoidal(grid.B_NAMES), "species": [],
          "rho": np.zeros(shape)}
    W0 = diagnostics.field_energy(st["E"], st["B"], dx)
    for _ in range(40):
        step.hybrid_step(p, st)
    W1 = diagnostics.field_energy(st["E"], st["B"], dx)
    assert abs(W1 - W0) < 1e-12 * W0


def test_cold_plasma_oscillation_at_plasma_frequency():
    # Langmuir oscillation: n0 = 1, q = -1, m = 1, eps0 = 1 -> omega_p = 1 (textbook).
    shape, dx, dt, ppc = (2, 2, 32), (1.0, 1.0, 1.0), 0.1, 4
    L = shape[2] * dx[2]
    kz = 2 * np.pi / L
    n = shape[0] * shape[1] * shape[2] * ppc
    rng = np.random.default_rng(0)
    z0 = (np.arange(n) + 0.5) * L / n
    x = rng.uniform(0, shape[0] * dx[0], n)
    y = rng.uniform(0, shape[1] * dx[1], n)
    A = 0.02
    z = np.mod(z0 + A * np.sin(kz * z0), L)
    dV = np.prod(dx)
    w = np.full(n, shape[0] * shape[1] * shape[2] * dV / n)
    sp = {"x": x, "y": y, "z": z, "ux": np.zeros(n), "uy": np.zeros(n), "uz": np.zeros(n),
          "w": w, "q": -1.0, "m": 1.0}
    p = step.Params(shape, dx, dt, 1, (8, 8, 8))
    rho = step.initial_rho(p, [sp])
    # E consistent with Gauss's law on the staggered grid: [k]_s . E = -i rho / eps0
    k = psatd.staggered_k_grid(shape, dx, (0, 0, 0))
    k2 = sum(k[a] ** 2 for a in range(3))
    rh = grid.to_spectral(rho, "rho", dx)
    E = [grid.from_spectral(np.where(k2 == 0, 0, -1j * rh * k[a] / np.where(k2 == 0, 1, k2)),
                            grid.E_NAMES[a], dx)[0] for a in range(3)]
    st = {"E": E, "B": [np.zeros(shape) for _ in range(3)], "species": [sp], "rho": rho}
    series = []
    for _ in range(140):
        step.hybrid_step(p, st)
        series.append(np.mean(st["E"][2][:, :, :] * np.sin(kz * (np.arange(shape[2]) + 0.5) * dx[2])))
    s = np.array(series)
    t = (np.arange(len(s)) + 1) * dt
    crossings = t[:-1][np.sign(s[:-1]) != np.sign(s[1:])]
    period = 2 * np.mean(np.diff(crossings))
    omega = 2 * np.pi / period
    assert abs(omega - 1.0) < 0.03


@pytest.mark.parametrize("variant,order,v", [(0, (8, 8, 8), 0.0), (1, (16, 16, 16), 0.9)])
def test_nodal_cycle_vacuum_energy_conserved(variant, order, v):
    # the nodal comparison cycle (Sec. 2): all quantities on the nodes, [k]_c in the solver
    shape, dx, dt = (8, 8, 16), (1.0, 0.8, 0.5), 0.45
    p = step.Params(shape, dx, dt, 1, (8, 8, 8), variant, (0.0, 0.0, v), order, cycle=step.NODAL)
    rng = np.random.default_rng(1)
    k = psatd.staggered_k_grid(shape, dx, order, nodal=True)
    k2 = sum(k[a] ** 2 for a in range(3))
    k2s = np.where(k2 == 0, 1.0, k2)

    def solenoidal():
        F = [np.fft.fftn(rng.normal(size=shape)) for _ in range(3)]
        kd = sum(k[a] * F[a] for a in range(3)) / k2s
        return [np.fft.ifftn(F[a] - k[a] * kd).real for a in range(3)]

    st = {"E": solenoidal(), "B": solenoidal(), "species": [], "rho": np.zeros(shape)}
    W0 = diagnostics.field_energy(st["E"], st["B"], dx)
    for _ in range(40):
        step.hybrid_step(p, st)
    W1 = diagnostics.field_energy(st["E"], st["B"], dx)
    assert abs(W1 - W0) < 1e-12 * W0


def test_nodal_and_staggered_dispersion_at_nyquist():
    # Sec. 2 (i): at finite order the nodal solver's vacuum waves stand still at the Nyquist
    # wave number ([k]_c = 0 there), the staggered solver's do not; omega = c |[k]_c| / c |[k]_s|
    from oracle import fornberg
    shape, dx, dt, order = (4, 4, 32), (1.0, 1.0, 1.0), 0.5, (16, 16, 16)
    N = shape[2]
    for nodal in (False, True):
        co = psatd.coefficients(shape, dx, dt, order, nodal=nodal)
        kk = psatd.staggered_k_grid(shape, dx, order, nodal=nodal)
        w = diagnostics.vacuum_dispersion(co, kk, 2, 1.0, dt)
        ref = fornberg.k_centered(N, 1.0, 16) if nodal else fornberg.k_staggered(N, 1.0, 16)
        np.testing.assert_allclose(w, np.abs(np.asarray(ref, np.float64)), rtol=1e-12, atol=1e-13)
        nyq = N // 2
        assert (w[nyq] < 1e-12) if nodal else (w[nyq] > 1.0)


def test_nodal_cycle_charge_conserved():
    w = workloads.thermal_plasma(shape=(8, 8, 8), ppc=2)
    p = step.Params(**w["params"], cycle=step.NODAL)
    st = {"E": [a.copy() for a in w["E"]], "B": [a.copy() for a in w["B"]],
          "species": [dict(s) for s in w["species"]]}
    st["rho"] = step.initial_rho(p, st["species"])
    qtot = sum(float(np.sum(s["q"] * s["w"])) for s in st["species"])
    qabs = sum(float(np.sum(np.abs(s["q"] * s["w"]))) for s in st["species"])
    for _ in range(3):
        step.hybrid_step(p, st)
        assert abs(np.sum(st["rho"]) * np.prod(p.dx) - qtot) < 1e-12 * qabs
        assert st["max_imag"] < 1e-9 * max(1.0, max(np.abs(e).max() for e in st["E"]))


def test_staggered_cycle_charge_conserved_and_real():
    w = workloads.laser_wakefield(shape=(8, 8, 32), ppc=1)
    p = step.Params(**w["params"], cycle=step.STAGGERED)
    st = {"E": [a.copy() for a in w["E"]], "B": [a.copy() for a in w["B"]],
          "species": [dict(s) for s in w["species"]]}
    st["rho"] = step.initial_rho(p, st["species"])
    qtot = sum(float(np.sum(s["q"] * s["w"])) for s in st["species"])
    qabs = sum(float(np.sum(np.abs(s["q"] * s["w"]))) for s in st["species"])
    for _ in range(3):
        step.hybrid_step(p, st)
        assert abs(np.sum(st["rho"]) * np.prod(p.dx) - qtot) < 1e-12 * qabs
        assert st["max_imag"] < 1e-9 * max(1.0, max(np.abs(e).max() for e in st["E"]))
