"""The synthetic inputs (paper_2106_12919_gb300/workloads.py) against the configurations they stand
in for: grid, spacings, time step, shape and centering orders, solver variant, particles per cell,
weights, momentum distributions, the laser and seed-wave profiles and the driver beam's moments."""
import numpy as np

from paper_2106_12919_gb300 import workloads


def _per_cell(sp, shape, dx):
    c = [np.floor(sp[k] / dx[a]).astype(np.int64) for a, k in enumerate("xyz")]
    return np.bincount((c[0] * shape[1] + c[1]) * shape[2] + c[2], minlength=int(np.prod(shape)))


def test_thermal_plasma():
    w = workloads.thermal_plasma()
    p = w["params"]
    assert p["shape"] == (32, 32, 32) and p["dx"] == (1.0, 1.0, 1.0) and p["dt"] == 1.0
    assert p["shape_order"] == 1 and p["centering_order"] == (8, 8, 8) and p["spectral_order"] == (0, 0, 0)
    assert p["variant"] == workloads.STANDARD
    (s,) = w["species"]
    assert s["x"].size == 262144 and s["q"] == -1.0 and s["m"] == 1.0
    assert np.all(_per_cell(s, p["shape"], p["dx"]) == 8)
    assert np.allclose(s["w"], 1.0 / 8)                        # n dV / ppc with n = 1
    for k in ("ux", "uy", "uz"):
        assert abs(np.std(s[k]) - 0.01) < 3e-4 and abs(np.mean(s[k])) < 1e-4
    assert all(np.all(a == 0) for a in w["E"] + w["B"])


def test_laser_wakefield():
    shape = (16, 16, 512)                                      # the full box's z length and physics
    w = workloads.laser_wakefield(shape=shape)
    p = w["params"]
    assert p["dx"] == (0.2, 0.2, 0.04) and p["dt"] == 0.04
    assert p["shape_order"] == 3 and p["centering_order"] == (8, 8, 16) and p["variant"] == workloads.STANDARD
    (s,) = w["species"]
    dz = p["dx"][2]
    assert np.all(_per_cell(s, shape, p["dx"]) == 2)
    dV = np.prod(p["dx"])
    assert np.allclose(s["w"], np.minimum(1.0, s["z"] / (50 * dz)) * dV / 2)   # 50-cell up-ramp
    assert all(np.all(s[k] == 0) for k in ("ux", "uy", "uz"))                 # cold
    Ey, Bx = w["E"][1], w["B"][0]
    k0 = 2 * np.pi / (30 * dz)
    assert abs(np.abs(Ey).max() / (2.0 * k0) - 1) < 0.01                     # a0 omega0, a0 = 2
    assert abs(np.abs(Bx).max() / np.abs(Ey).max() - 1) < 0.01
    # envelope centred 150 cells into the box, Gaussian length 60 cells
    env = np.abs(Ey).max(axis=(0, 1))
    assert abs(int(np.argmax(env)) - 150) <= 8
    assert env[150 + 60] < 0.45 * env.max() and env[150 + 30] > 0.6 * env.max()
    assert np.all(w["E"][0] == 0) and np.all(w["E"][2] == 0)


def test_galilean_drift():
    w = workloads.galilean_drift(shape=(8, 8, 32))
    p = w["params"]
    gamma = 130.0
    beta = np.sqrt(1 - 1 / gamma ** 2)
    assert p["variant"] == workloads.GALILEAN and p["v_gal"] == (0.0, 0.0, beta)
    assert p["spectral_order"] == (16, 16, 16) and p["shape_order"] == 2 and p["centering_order"] == (8, 8, 8)
    e, pos = w["species"]
    assert e["q"] == -1.0 and pos["q"] == 1.0
    for k in "xyz":
        assert np.array_equal(e[k], pos[k])                    # co-located pairs
    assert np.all(_per_cell(e, p["shape"], p["dx"]) == 2)
    for s in (e, pos):
        assert abs(np.mean(s["uz"]) - gamma * beta) < 1e-3 and abs(np.std(s["ux"]) - 1e-3) < 1e-4
    assert not np.array_equal(e["ux"], pos["ux"])              # independent momenta


def test_seed_wave_and_probe():
    shape = (32, 32, 64)
    A = 0.01
    w = workloads.seed_wave(shape=shape, amplitude=A)
    p = w["params"]
    assert p["shape_order"] == 1 and p["centering_order"] == (8, 8, 8) and p["variant"] == workloads.STANDARD
    (s,) = w["species"]
    assert np.all(_per_cell(s, shape, p["dx"]) == 4)
    assert abs(np.std(s["ux"]) - 0.05) < 2e-3
    z = np.arange(shape[2]) + 0.0                               # E_x sits at (i + 1/2, j, k)
    want = A * np.exp(-((z - shape[2] / 2) / 8.0) ** 2) * np.cos(2 * np.pi * z / 16.0)
    assert np.allclose(w["E"][0][3, 5, :], want, atol=1e-15)
    lo, hi = w["probe"]
    assert all(hi[a] - lo[a] == 16 and lo[a] + hi[a] == shape[a] for a in range(3))   # central 16^3


def test_beam_wakefield_driver():
    shape = (32, 32, 128)
    nb = 40000
    w = workloads.beam_wakefield(shape=shape, n_beam=nb)
    p = w["params"]
    dx = p["dx"]
    gamma = 1000.0
    assert dx == (0.1, 0.1, 0.02) and p["dt"] == 0.02 and p["variant"] == workloads.AVERAGED
    assert p["v_gal"] == (0.0, 0.0, np.sqrt(1 - 1 / gamma ** 2)) and p["centering_order"] == (8, 8, 16)
    plasma, beam = w["species"]
    assert np.all(_per_cell(plasma, shape, dx) == 1)
    L = [shape[a] * dx[a] for a in range(3)]
    for a, k in enumerate("xyz"):
        centre = (0.5, 0.5, 0.75)[a] * L[a]
        sigma = (4 * dx[0], 4 * dx[1], 10 * dx[2])[a]
        d = np.mod(beam[k] - centre + 0.5 * L[a], L[a]) - 0.5 * L[a]    # periodic: tails wrap around
        assert abs(np.mean(d)) < 0.02 * sigma
        assert abs(np.std(d) / sigma - 1) < 0.02
    assert np.allclose(beam["uz"], np.sqrt(gamma ** 2 - 1)) and np.all(beam["ux"] == 0)
    # peak density of the Gaussian driver: sum w / ((2 pi)^(3/2) sigma_x sigma_y sigma_z) = 10 n0
    peak = beam["w"].sum() / ((2 * np.pi) ** 1.5 * (4 * dx[0]) ** 2 * 10 * dx[2])
    assert abs(peak - 10.0) < 1e-12
