"""GPU parity of the particle rows: tile binning, gather + Boris + move + deposit,
and the initial charge deposition (libpic through the C ABI vs the oracle)."""
import numpy as np
import pytest

from helpers import TOL, context_for, field_rel_err, periodic_pos_err, species_from_dev, species_to_dev, to_dev, to_host
from oracle import particles
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu


def _rand_species(rng, n, shape, dx, q=-1.0, m=1.0, u=0.3):
    L = [shape[a] * dx[a] for a in range(3)]
    return {"x": rng.uniform(0, L[0], n), "y": rng.uniform(0, L[1], n), "z": rng.uniform(0, L[2], n),
            "ux": rng.normal(0, u, n), "uy": rng.normal(0, u, n), "uz": rng.normal(0, u, n),
            "w": rng.uniform(0.5, 1.5, n), "q": q, "m": m}


@pytest.mark.parametrize("shape,tile,n", [((16, 8, 32), (8, 8, 8), 5000), ((32, 32, 64), (8, 4, 16), 100000),
                                          ((8, 8, 16), (8, 8, 16), 777), ((16, 16, 16), (2, 2, 2), 0)])
def test_bin_offsets_exact(shape, tile, n):
    import torch
    dx = (0.5, 1.0, 0.25)
    p = dict(shape=shape, dx=dx, dt=0.1, shape_order=1, centering_order=(2, 2, 2), variant=0,
             v_gal=(0, 0, 0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)
    ctx = context_for(p, tile=tile)
    rng = np.random.default_rng(n)
    sp = _rand_species(rng, n, shape, dx)
    tid, off_ref, _ = particles.tile_bins([sp["x"], sp["y"], sp["z"]], dx, shape, tile)
    (dsp,) = species_to_dev([sp])
    off = torch.empty(ctx.num_tiles() + 1, dtype=torch.int64, device="cuda")
    ctx.bin(dsp, off)
    ctx.sync()
    np.testing.assert_array_equal(to_host(off), off_ref)          # bit-exact offsets
    ids = to_host(dsp.id)
    assert np.array_equal(np.sort(ids), np.arange(n))             # a permutation
    np.testing.assert_array_equal(to_host(dsp.x), sp["x"][ids])   # arrays moved together
    np.testing.assert_array_equal(to_host(dsp.w), sp["w"][ids])
    assert np.all(np.diff(tid[ids]) >= 0)                         # tile ids non-decreasing


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("variant,v", [(0, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 0.9)), (2, (0.3, -0.2, 0.5))])
def test_push_deposit(order, variant, v):
    import torch
    shape, dx, dt = (16, 8, 32), (0.5, 1.0, 0.25), 0.2
    p = dict(shape=shape, dx=dx, dt=dt, shape_order=order, centering_order=(4, 4, 4), variant=variant,
             v_gal=v, spectral_order=(0, 0, 0), c=1.0, eps0=1.0)
    ctx = context_for(p)
    rng = np.random.default_rng(order)
    sp = [_rand_species(rng, 3000, shape, dx), _rand_species(rng, 1000, shape, dx, q=2.0, m=3.0)]
    En = [rng.normal(size=shape) for _ in range(3)]
    Bn = [rng.normal(size=shape) for _ in range(3)]
    Jref = [np.zeros(shape) for _ in range(3)]
    rho_ref = np.zeros(shape)
    new_ref = []
    for s in sp:
        ns, J, r = particles.push_and_deposit(s, En, Bn, shape, dx, dt, order, v)
        new_ref.append(ns)
        for a in range(3):
            Jref[a] += J[a]
        rho_ref += r
    dsp = species_to_dev(sp)
    Jd = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    rd = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
    ctx.push_deposit([to_dev(a) for a in En], [to_dev(a) for a in Bn], dsp, Jd, rd)
    ctx.sync()
    assert field_rel_err([to_host(a).reshape(shape) for a in Jd], Jref) < TOL
    assert field_rel_err([to_host(rd).reshape(shape)], [rho_ref]) < TOL
    L = [shape[a] * dx[a] for a in range(3)]
    for g, r in zip(species_from_dev(dsp), new_ref):
        for a, k in enumerate(("x", "y", "z")):
            assert np.max(periodic_pos_err(g[k], r[k], L[a])) < 1e-12 * L[a]
        for k in ("ux", "uy", "uz"):
            assert np.max(np.abs(g[k] - r[k])) < 1e-12 * np.max(np.abs(r[k]))


def test_deposit_rho_charge():
    import torch
    w = workloads.laser_wakefield(shape=(16, 16, 64), ppc=1)
    p = w["params"]
    ctx = context_for(p)
    from oracle import step
    ref = step.initial_rho(step.Params(**p), w["species"])
    rd = torch.empty(ctx.ncell, dtype=torch.float64, device="cuda")
    ctx.deposit_rho(species_to_dev(w["species"]), rd)
    assert field_rel_err([to_host(rd).reshape(p["shape"])], [ref]) < TOL
    q = ctx.total_charge(rd)
    qtot = sum(np.sum(s["q"] * s["w"]) for s in w["species"])
    assert abs(q - qtot) < 1e-12 * abs(qtot)
