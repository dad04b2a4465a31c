"""Parity at the benchmark's full size (laser-wakefield box, 128 x 128 x 512 cells,
16,777,216 particles), in the launch configuration bench.py times.

* Field solve: the whole-grid Maxwell step of the oracle (numpy FFTs, long-double
  coefficients) against pic_maxwell_step on the full box, 1e-12.
* Particles: a sample of 256 particles is pushed by the oracle one by one from the
  inputs (its own real-space centering of the input E, B, then gather, Boris and
  move) and compared with the particles after one pic_step / pic_step32.
* Charge: total deposited charge equals sum q w (a property at any size).
"""
import numpy as np
import pytest

from helpers import TOL, context_for, field_rel_err, periodic_pos_err, to_dev, to_host
from oracle import grid, particles, step
from paper_2106_12919_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FULL = (128, 128, 512)


@pytest.fixture(scope="module")
def wf():
    return workloads.laser_wakefield(shape=FULL)


def test_fullsize_field_solve_fp64(wf):
    p = wf["params"]
    ctx = context_for(p)
    op = step.Params(**p)
    rng = np.random.default_rng(21)
    J = [1e-3 * rng.normal(size=FULL) for _ in range(3)]
    rn = 1e-3 * rng.normal(size=FULL)
    rp = rn + 1e-4 * rng.normal(size=FULL)
    Eo, Bo, _, _ = step.maxwell_update(op, wf["E"], wf["B"], J, rn, rp)
    Ed, Bd = [to_dev(a) for a in wf["E"]], [to_dev(a) for a in wf["B"]]
    ctx.maxwell_step(Ed, Bd, [to_dev(a) for a in J], to_dev(rn), to_dev(rp))
    ctx.sync()
    assert field_rel_err([to_host(a).reshape(FULL) for a in Ed], Eo) < TOL
    assert field_rel_err([to_host(a).reshape(FULL) for a in Bd], Bo) < TOL


def _oracle_sample_push(wf, idx):
    """Oracle push of the sampled particles from the input fields (real-space centering)."""
    p = wf["params"]
    o = p["centering_order"]
    nE = [grid.center_to_nodal(wf["E"][a], grid.E_NAMES[a], o) for a in range(3)]
    nB = [grid.center_to_nodal(wf["B"][a], grid.B_NAMES[a], o) for a in range(3)]
    s = wf["species"][0]
    sub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    pos = [sub["x"], sub["y"], sub["z"]]
    E = particles.gather(nE, pos, p["dx"], p["shape_order"])
    B = particles.gather(nB, pos, p["dx"], p["shape_order"])
    u = particles.boris([sub["ux"], sub["uy"], sub["uz"]], E, B, sub["q"], sub["m"], p["dt"], p["c"])
    g = np.sqrt(1.0 + (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / p["c"] ** 2)
    L = [FULL[a] * p["dx"][a] for a in range(3)]
    new = [particles.wrap(pos[a] + p["dt"] * u[a] / g, L[a]) for a in range(3)]
    return new, u


def _sample(n):
    # particles with a field acting on them: spread over the box, plus the laser region
    rng = np.random.default_rng(5)
    return np.unique(np.concatenate([rng.integers(0, n, 128),
                                     np.arange(n // 2, n // 2 + 2 * 512 * 128, 1024)[:128]]))


def test_fullsize_sampled_particles_and_charge_fp64(wf):
    import torch
    from helpers import species_to_dev
    p = wf["params"]
    ctx = context_for(p)
    s = wf["species"][0]
    n = s["x"].size
    idx = _sample(n)
    new_ref, u_ref = _oracle_sample_push(wf, idx)
    (sp,) = species_to_dev(wf["species"])
    E, B = [to_dev(a) for a in wf["E"]], [to_dev(a) for a in wf["B"]]
    J = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    rho = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
    ctx.deposit_rho([sp], rho)
    ctx.step(E, B, J, rho, [sp], 1)
    ctx.sync()
    ids = to_host(sp.id)
    where = np.empty(n, dtype=np.int64)
    where[ids] = np.arange(n)
    L = [FULL[a] * p["dx"][a] for a in range(3)]
    for a, k in enumerate(("x", "y", "z")):
        got = to_host(getattr(sp, k))[where[idx]]
        assert np.max(periodic_pos_err(got, new_ref[a], L[a])) < 1e-12 * L[a]
    for a, k in enumerate(("ux", "uy", "uz")):
        got = to_host(getattr(sp, k))[where[idx]]
        scale = max(np.max(np.abs(u_ref[a])), 1e-30)
        assert np.max(np.abs(got - u_ref[a])) < 1e-12 * scale, k
    q = ctx.total_charge(rho)
    qtot = float(np.sum(s["q"] * s["w"]))
    assert abs(q - qtot) < 1e-12 * abs(qtot)


def test_fullsize_sampled_particles_and_charge_fp32(wf):
    import torch
    from paper_2106_12919_gb300 import pic
    p = wf["params"]
    ctx = context_for(p, precision=pic.PIC_FP32)
    s = wf["species"][0]
    n = s["x"].size
    sp = pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"], s["q"], s["m"],
                                      id=torch.arange(n, dtype=torch.int64, device="cuda"))
    # the oracle starts from the same particle set: positions as the FP32 form holds them
    x0 = sp.positions(ctx)
    wf32 = dict(wf)
    wf32["species"] = [dict(s, x=x0[0], y=x0[1], z=x0[2])]
    wf32["E"] = [a.astype(np.float32).astype(np.float64) for a in wf["E"]]
    wf32["B"] = [a.astype(np.float32).astype(np.float64) for a in wf["B"]]
    idx = _sample(n)
    new_ref, u_ref = _oracle_sample_push(wf32, idx)
    E = [torch.from_numpy(a.astype(np.float32)).cuda() for a in wf["E"]]
    B = [torch.from_numpy(a.astype(np.float32)).cuda() for a in wf["B"]]
    J = [torch.empty(ctx.ncell, dtype=torch.float32, device="cuda") for _ in range(3)]
    rho = torch.empty(ctx.ncell, dtype=torch.float32, device="cuda")
    ctx.deposit_rho32([sp], rho)
    ctx.step32(E, B, J, rho, [sp], 1)
    ctx.sync()
    ids = to_host(sp.id)
    where = np.empty(n, dtype=np.int64)
    where[ids] = np.arange(n)
    pos = sp.positions(ctx)
    L = [FULL[a] * p["dx"][a] for a in range(3)]
    for a in range(3):
        assert np.max(periodic_pos_err(pos[a][where[idx]], new_ref[a], L[a])) < 2e-6 * L[a] / FULL[a] * 8
    for a, k in enumerate(("ux", "uy", "uz")):
        got = to_host(getattr(sp, k)).astype(np.float64)[where[idx]]
        scale = max(np.max(np.abs(u_ref[a])), 1e-30)
        assert np.max(np.abs(got - u_ref[a])) < 2e-6 * scale, k
    q = ctx.total_charge32(rho)
    qtot = float(np.sum(s["q"] * s["w"].astype(np.float32).astype(np.float64)))
    assert abs(q - qtot) < 1e-5 * abs(qtot)
