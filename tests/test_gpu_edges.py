"""Edge cases of the particle path, GPU against the oracle through the C ABI: empty species,
ragged particle counts (1, 31, 257 and one more than a chunk of the tiled push), particles on cell
faces and at the ends of the periodic box, and tiles whose particle count sits on either side of
the tiled push's chunk size (2048)."""
import numpy as np
import pytest

from helpers import TOL, context_for, field_rel_err, periodic_pos_err, species_from_dev, species_to_dev, to_dev, to_host
from oracle import particles, step
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu

CHUNK = 2048


def _params(shape=(16, 8, 32), dx=(0.5, 1.0, 0.25), dt=0.2, order=3):
    return dict(shape=shape, dx=dx, dt=dt, shape_order=order, centering_order=(4, 4, 4), variant=0,
                v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)


def _species(rng, n, shape, dx, x=None, y=None, z=None):
    L = [shape[a] * dx[a] for a in range(3)]
    return {"x": rng.uniform(0, L[0], n) if x is None else x, "y": rng.uniform(0, L[1], n) if y is None else y,
            "z": rng.uniform(0, L[2], n) if z is None else z, "ux": rng.normal(0, 0.3, n),
            "uy": rng.normal(0, 0.3, n), "uz": rng.normal(0, 0.3, n), "w": rng.uniform(0.5, 1.5, n),
            "q": -1.0, "m": 1.0}


def _push_parity(p, sp_list, rng):
    import torch
    shape, dx = p["shape"], p["dx"]
    ctx = context_for(p)
    En = [rng.normal(size=shape) for _ in range(3)]
    Bn = [rng.normal(size=shape) for _ in range(3)]
    Jref = [np.zeros(shape) for _ in range(3)]
    rref = np.zeros(shape)
    new = []
    for s in sp_list:
        ns, J, r = particles.push_and_deposit(s, En, Bn, shape, dx, p["dt"], p["shape_order"])
        new.append(ns)
        for a in range(3):
            Jref[a] += J[a]
        rref += r
    dsp = species_to_dev(sp_list)
    Jd = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    rd = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
    ctx.push_deposit([to_dev(a) for a in En], [to_dev(a) for a in Bn], dsp, Jd, rd)
    ctx.sync()
    if any(s["x"].size for s in sp_list):
        assert field_rel_err([to_host(a).reshape(shape) for a in Jd], Jref) < TOL
        assert field_rel_err([to_host(rd).reshape(shape)], [rref]) < TOL
    else:
        assert all(float(t.abs().max()) == 0.0 for t in Jd + [rd])
    L = [shape[a] * dx[a] for a in range(3)]
    for g, r in zip(species_from_dev(dsp), new):
        for a, k in enumerate(("x", "y", "z")):
            if r[k].size:
                assert np.max(periodic_pos_err(g[k], r[k], L[a])) < 1e-12 * L[a]


@pytest.mark.parametrize("n", [0, 1, 31, 257, CHUNK + 1])
def test_push_deposit_ragged_counts(n):
    rng = np.random.default_rng(100 + n)
    p = _params()
    _push_parity(p, [_species(rng, n, p["shape"], p["dx"])], rng)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_particles_on_faces_and_box_ends(order):
    """Positions on cell faces (integer multiples of dx), at 0 and at the last representable
    position below L (the periodic wrap), for every shape order."""
    rng = np.random.default_rng(7 + order)
    p = _params(order=order)
    shape, dx = p["shape"], p["dx"]
    L = [shape[a] * dx[a] for a in range(3)]
    faces = [np.concatenate([np.arange(shape[a]) * dx[a], [0.0, np.nextafter(L[a], 0.0), dx[a] * 0.5]])
             for a in range(3)]
    n = 600
    pick = [rng.choice(faces[a], n) for a in range(3)]
    sp = _species(rng, n, shape, dx, *pick)
    _push_parity(p, [sp], rng)


@pytest.mark.parametrize("fp32", [False, True])
def test_step_with_an_empty_species(fp32):
    """An empty species beside a full one changes nothing (both forms, tiled FP32 push)."""
    import torch
    from paper_2106_12919_gb300 import pic
    w = workloads.thermal_plasma(shape=(16, 16, 16), ppc=2)
    p = w["params"]
    shape, dx = p["shape"], p["dx"]
    empty = {k: (v[:0].copy() if isinstance(v, np.ndarray) else v) for k, v in w["species"][0].items()}
    outs = []
    for with_empty in (False, True):
        sps = w["species"] + ([empty] if with_empty else [])
        if fp32:
            ctx = context_for(p, sort_interval=2, precision=pic.PIC_FP32)
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
            sp = [pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                               s["q"], s["m"]) for s in sps]
            E, B = [dev(a) for a in w["E"]], [dev(a) for a in w["B"]]
            rho = torch.empty(ctx.ncell, dtype=torch.float32, device="cuda")
            ctx.deposit_rho32(sp, rho)
            ctx.step32(E, B, None, rho, sp, 3)
        else:
            ctx = context_for(p, sort_interval=2)
            sp = species_to_dev(sps)
            E, B = [to_dev(a) for a in w["E"]], [to_dev(a) for a in w["B"]]
            rho = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
            ctx.deposit_rho(sp, rho)
            ctx.step(E, B, None, rho, sp, 3)
        ctx.sync()
        outs.append([to_host(t).astype(np.float64) for t in E + B + [rho]])
    assert field_rel_err(outs[1], outs[0]) < (1e-6 if fp32 else 1e-13)


def test_tiled_push_chunk_boundaries():
    """Tiles holding CHUNK - 1, CHUNK, CHUNK + 1 and 2 CHUNK + 1 particles (one, one, two and three
    chunks of the tiled FP32 push) and empty tiles: one FP32 step against the FP64 oracle."""
    import torch
    from paper_2106_12919_gb300 import pic
    shape, dx, dt = (16, 16, 32), (1.0, 1.0, 1.0), 0.5
    p = dict(shape=shape, dx=dx, dt=dt, shape_order=3, centering_order=(4, 4, 4), variant=0,
             v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)
    rng = np.random.default_rng(11)
    parts = []
    # tile origins (cells) with their particle counts; tiles are 8x8x8 cells
    for (tx, ty, tz), n in (((0, 0, 0), CHUNK - 1), ((8, 0, 8), CHUNK), ((0, 8, 16), CHUNK + 1),
                            ((8, 8, 24), 2 * CHUNK + 1)):
        parts.append([tx + rng.uniform(0.5, 7.5, n), ty + rng.uniform(0.5, 7.5, n), tz + rng.uniform(0.5, 7.5, n)])
    x, y, z = (np.concatenate([q[a] for q in parts]) for a in range(3))
    sp = _species(rng, x.size, shape, dx, x, y, z)
    sp["ux"] *= 0.1
    sp["uy"] *= 0.1
    sp["uz"] *= 0.1
    sp["w"] = np.full(x.size, 0.05)
    E0 = [rng.normal(size=shape) * 0.1 for _ in range(3)]
    B0 = [np.zeros(shape) for _ in range(3)]
    ctx = context_for(p, sort_interval=1, precision=pic.PIC_FP32)
    (d,) = [pic.Species32.from_positions(ctx, sp["x"], sp["y"], sp["z"], sp["ux"], sp["uy"], sp["uz"], sp["w"],
                                         sp["q"], sp["m"], id=torch.arange(x.size, dtype=torch.int64, device="cuda"))]
    # the oracle gets the same (cell, FP32 offset) particles in FP64
    order = np.argsort(to_host(d.id))
    px, py, pz = d.positions(ctx)
    ref_sp = {"x": px[order], "y": py[order], "z": pz[order], "q": sp["q"], "m": sp["m"]}
    for k in ("ux", "uy", "uz", "w"):
        ref_sp[k] = to_host(getattr(d, k)).astype(np.float64)[order]
    E32 = [a.astype(np.float32).astype(np.float64) for a in E0]
    op = step.Params(**p)
    st = {"E": [a.copy() for a in E32], "B": [a.copy() for a in B0], "species": [ref_sp]}
    st["rho"] = step.initial_rho(op, st["species"])
    for _ in range(2):
        step.hybrid_step(op, st)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    E, B = [dev(a) for a in E32], [dev(a) for a in B0]
    J = [torch.empty(ctx.ncell, dtype=torch.float32, device="cuda") for _ in range(3)]
    rho = torch.empty(ctx.ncell, dtype=torch.float32, device="cuda")
    ctx.deposit_rho32([d], rho)
    ctx.step32(E, B, J, rho, [d], 2)
    ctx.sync()
    g = lambda ts: [to_host(t).astype(np.float64).reshape(shape) for t in ts]
    assert field_rel_err(g(J), st["J"]) < 1e-5
    assert field_rel_err(g([rho]), [st["rho"]]) < 1e-5
    assert field_rel_err(g(E), st["E"]) < 1e-5
    # every particle is still there, once
    ids = to_host(d.id)
    assert np.array_equal(np.sort(ids), np.arange(x.size))
