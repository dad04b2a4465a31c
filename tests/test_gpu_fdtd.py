"""GPU parity of the hybrid FDTD cycle (PIC_CYCLE_HYBRID_FDTD: the hybrid scheme around a Yee
finite-difference solver of order 2m, the adaptation to FDTD of Sec. 6) against the oracle's
cycle (oracle/step.py with oracle/fdtd.py), FP64, through the C ABI.

Tolerance 1e-12 relative (L2 per field).  dt is set to 0.9 of each case's Courant limit (the
workloads' own dt = dx is above the 3D Yee limit)."""
import numpy as np
import pytest

from helpers import TOL, context_for, field_rel_err, periodic_pos_err, species_from_dev, species_to_dev, to_dev, to_host
from oracle import fdtd, fornberg, step
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu

FDTD = 3

# (workload, generator args, steps, finite-difference order per axis (0 = Yee's order 2), options)
CASES = [
    ("thermal_plasma", dict(shape=(16, 16, 16), ppc=4), 4, (0, 0, 0), {}),
    ("thermal_plasma", dict(shape=(16, 16, 16), ppc=4), 4, (4, 8, 2), {}),
    ("laser_wakefield", dict(shape=(16, 16, 64), ppc=1), 3, (0, 0, 0), {}),
    ("laser_wakefield", dict(shape=(16, 16, 64), ppc=1), 3, (4, 4, 16), {}),
    ("seed_wave", dict(shape=(16, 16, 16), ppc=2), 3, (2, 2, 2), {}),
    # the bilinear smoothing of J (Sec. 2) and Vay's pusher around the FDTD solver
    ("thermal_plasma", dict(shape=(16, 16, 16), ppc=4), 4, (0, 0, 0), {"filter_passes": 2}),
    ("laser_wakefield", dict(shape=(16, 16, 64), ppc=1), 3, (4, 4, 8), {"filter_passes": 1, "pusher": 1}),
]


def _params(w, orders):
    p = dict(w["params"])
    p["spectral_order"] = orders
    p["dt"] = 0.9 * fdtd.courant_limit(tuple(o or 2 for o in orders), p["dx"], p["c"])
    return p


def _rng_fields(shape, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=shape) for _ in range(3)]


@pytest.mark.parametrize("orders", [(0, 0, 0), (4, 2, 8), (16, 16, 16)])
def test_maxwell_step_matches_yee_update(orders):
    import torch
    shape, dx = (16, 32, 64), (0.5, 0.7, 0.3)
    lim = fdtd.courant_limit(tuple(o or 2 for o in orders), dx, 1.3)
    p = dict(shape=shape, dx=dx, dt=0.8 * lim, shape_order=1, centering_order=(8, 8, 8), variant=0,
             v_gal=(0.0, 0.0, 0.0), spectral_order=orders, c=1.3, eps0=0.7)
    ctx = context_for(p, cycle=FDTD)
    E, B, J = _rng_fields(shape, 1), _rng_fields(shape, 2), _rng_fields(shape, 3)
    dE, dB, dJ = [to_dev(a) for a in E], [to_dev(a) for a in B], [to_dev(a) for a in J]
    ctx.maxwell_step(dE, dB, dJ, None, None)
    ctx.sync()
    fo = tuple(o or 2 for o in orders)
    rE, rB = fdtd.yee_update(E, B, J, p["dt"], fo, dx, 1.3, 0.7)
    g = lambda ts: [to_host(t).reshape(shape) for t in ts]
    assert field_rel_err(g(dE), rE) < TOL
    assert field_rel_err(g(dB), rB) < TOL
    # J is read only
    assert field_rel_err(g(dJ), J) == 0.0


@pytest.mark.parametrize("name,kw,nsteps,orders,opts", CASES)
def test_fdtd_cycle_matches_oracle(name, kw, nsteps, orders, opts):
    import torch
    w = workloads.WORKLOADS[name](**kw)
    p = _params(w, orders)
    shape = p["shape"]
    prm = step.Params(**p, cycle=FDTD, **opts)
    st = {"E": [a.copy() for a in w["E"]], "B": [a.copy() for a in w["B"]],
          "species": [dict(s) for s in w["species"]]}
    st["rho"] = step.initial_rho(prm, st["species"])
    for _ in range(nsteps):
        step.hybrid_step(prm, st)
    ctx = context_for(p, sort_interval=2, cycle=FDTD, **opts)
    E = [to_dev(a) for a in w["E"]]
    B = [to_dev(a) for a in w["B"]]
    J = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    rho = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
    sp = species_to_dev(w["species"])
    ctx.deposit_rho(sp, rho)
    ctx.step(E, B, J, rho, sp, nsteps)
    ctx.sync()
    g = lambda ts: [to_host(t).reshape(shape) for t in ts]
    assert field_rel_err(g(E), st["E"]) < TOL
    assert field_rel_err(g(B), st["B"]) < TOL
    assert field_rel_err(g(J), st["J"]) < TOL
    assert field_rel_err(g([rho]), [st["rho"]]) < TOL
    L = [shape[a] * p["dx"][a] for a in range(3)]
    for gs, rs in zip(species_from_dev(sp), st["species"]):
        for a, k in enumerate(("x", "y", "z")):
            assert np.max(periodic_pos_err(gs[k], rs[k], L[a])) < 1e-11 * L[a]
        for k in ("ux", "uy", "uz"):
            scale = max(np.max(np.abs(rs[k])), 1e-300)
            assert np.linalg.norm(gs[k] - rs[k]) / max(np.linalg.norm(rs[k]), 1e-300) < TOL or \
                np.max(np.abs(gs[k] - rs[k])) < 1e-13 * scale


def test_split_calls_equal_one_call():
    """The FDTD state is the Yee E, B themselves: n calls of one step equal one call of n."""
    import torch
    w = workloads.thermal_plasma(shape=(16, 16, 16), ppc=2)
    p = _params(w, (0, 0, 0))
    outs = []
    for split in (False, True):
        ctx = context_for(p, sort_interval=0, cycle=FDTD)
        E = [to_dev(a) for a in w["E"]]
        B = [to_dev(a) for a in w["B"]]
        J = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
        rho = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
        sp = species_to_dev(w["species"])
        ctx.deposit_rho(sp, rho)
        if split:
            for _ in range(3):
                ctx.step(E, B, J, rho, sp, 1)
        else:
            ctx.step(E, B, J, rho, sp, 3)
        ctx.sync()
        outs.append([to_host(t) for t in E + B])
    assert field_rel_err(outs[1], outs[0]) < 1e-13


@pytest.mark.parametrize("orders", [(0, 0, 0), (4, 8, 2)])
def test_tables_and_dispersion(orders):
    """pic_axis_tables gives the difference's symbol [k]_s; pic_vacuum_dispersion the Yee relation
    sin(omega dt / 2) = c dt |[k]_s| / 2."""
    shape, dx, c = (16, 32, 64), (1.0, 0.5, 0.25), 1.0
    fo = tuple(o or 2 for o in orders)
    dt = 0.95 * fdtd.courant_limit(fo, dx, c)
    p = dict(shape=shape, dx=dx, dt=dt, shape_order=1, centering_order=(8, 8, 8), variant=0,
             v_gal=(0.0, 0.0, 0.0), spectral_order=orders, c=c, eps0=1.0)
    ctx = context_for(p, cycle=FDTD)
    for a in range(3):
        ks, _, _ = ctx.axis_tables(a)
        want = np.asarray(fornberg.k_staggered(shape[a], dx[a], fo[a]), dtype=np.float64)
        assert np.max(np.abs(np.asarray(ks) - want)) < 1e-14 * np.max(np.abs(want))
        om = np.asarray(ctx.vacuum_dispersion(a))
        wom = 2.0 * np.arcsin(0.5 * c * dt * np.abs(want)) / dt
        assert np.max(np.abs(om - wom)) < 1e-12 * np.max(wom)


def test_stable_just_below_the_courant_limit():
    """A vacuum run at 0.99 of the Courant limit keeps bounded fields (no growth of the
    Nyquist modes); the limit itself is refused above it (checked on the CPU in test_capi)."""
    import torch
    shape, dx = (16, 16, 16), (1.0, 1.0, 1.0)
    dt = 0.99 * fdtd.courant_limit((2, 2, 2), dx)
    p = dict(shape=shape, dx=dx, dt=dt, shape_order=1, centering_order=(2, 2, 2), variant=0,
             v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)
    ctx = context_for(p, cycle=FDTD)
    E = [to_dev(a * 1e-3) for a in _rng_fields(shape, 4)]
    B = [to_dev(np.zeros(shape)) for _ in range(3)]
    J = [torch.zeros(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    rho = torch.zeros(ctx.ncell, dtype=torch.float64, device="cuda")
    ctx.step(E, B, J, rho, [], 400)
    ctx.sync()
    amp = max(float(t.abs().max()) for t in E + B)
    assert np.isfinite(amp) and amp < 1.0
