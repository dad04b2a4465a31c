"""GPU parity of the diagnostics (stencil extent, axis tables, vacuum dispersion, beam RMS)
against the oracle, through the C ABI."""
import numpy as np
import pytest

from helpers import context_for, species_to_dev
from oracle import diagnostics, fornberg, psatd
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    # shape, dx, dt, spectral order, v_gal
    ((16, 8, 32), (0.5, 1.0, 0.25), 0.2, (0, 0, 0), (0.0, 0.0, 0.0)),
    ((16, 8, 32), (0.5, 1.0, 0.25), 0.2, (16, 8, 16), (0.0, 0.0, 0.0)),
    ((8, 16, 64), (1.0, 1.0, 1.0), 1.0, (8, 8, 16), (0.0, 0.0, 0.95)),
]


def _params(shape, dx, dt, order, v):
    return dict(shape=shape, dx=dx, dt=dt, shape_order=1, centering_order=(4, 6, 8),
                variant=1 if any(v) else 0, v_gal=v, spectral_order=order, c=1.0, eps0=1.0)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stencil_extent(case):
    shape, dx, dt, order, v = CASES[case]
    p = _params(shape, dx, dt, order, v)
    ctx = context_for(p)
    co = psatd.coefficients(shape, dx, dt, order, v)
    for name in ("TC", "TS", "X1", "X4"):
        for axis in range(3):
            ref = diagnostics.stencil_extent(co[name], axis)
            got = np.array(ctx.stencil_extent(name, axis))
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(ref), (name, axis)


def test_stencil_extent_rejects_bad_arguments():
    from paper_2106_12919_gb300 import pic
    ctx = context_for(_params(*CASES[0]))
    with pytest.raises(pic.PicError):
        ctx.stencil_extent("NOPE", 0)
    with pytest.raises(pic.PicError):
        ctx.stencil_extent("TC", 3)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_axis_tables(case):
    shape, dx, dt, order, v = CASES[case]
    p = _params(shape, dx, dt, order, v)
    ctx = context_for(p)
    for a in range(3):
        ks, kc, zt = (np.array(t) for t in ctx.axis_tables(a))
        np.testing.assert_allclose(ks, np.asarray(fornberg.k_staggered(shape[a], dx[a], order[a]), np.float64),
                                   rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(kc, np.asarray(fornberg.k_centered(shape[a], dx[a], order[a]), np.float64),
                                   rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(zt, np.asarray(fornberg.zeta(shape[a], p["centering_order"][a]),
                                                  np.float64), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_vacuum_dispersion(case):
    shape, dx, dt, order, v = CASES[case]
    p = _params(shape, dx, dt, order, v)
    ctx = context_for(p)
    co = psatd.coefficients(shape, dx, dt, order, v)
    k = psatd.staggered_k_grid(shape, dx, order)
    for axis in range(3):
        ref = diagnostics.vacuum_dispersion(co, k, axis, 1.0, dt)
        got = np.array(ctx.vacuum_dispersion(axis))
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))


def test_beam_rms_fp64_and_fp32():
    import torch
    from paper_2106_12919_gb300 import pic
    w = workloads.beam_wakefield(shape=(32, 32, 64), ppc=1, n_beam=20000)
    p = w["params"]
    beam = w["species"][1]
    ref = diagnostics.beam_rms(beam["x"], beam["y"], beam["w"])
    ctx = context_for(p)
    (sp,) = species_to_dev([beam], with_id=False)
    assert abs(ctx.beam_rms(sp) - ref) < 1e-12 * ref
    ctx32 = context_for(p, precision=pic.PIC_FP32)
    s32 = pic.Species32.from_positions(ctx32, beam["x"], beam["y"], beam["z"], beam["ux"], beam["uy"], beam["uz"],
                                       beam["w"], beam["q"], beam["m"])
    x, y, _ = s32.positions(ctx32)
    w32 = s32.w.cpu().numpy().astype(np.float64)
    ref32 = diagnostics.beam_rms(x, y, w32)
    assert abs(ctx32.beam_rms32(s32) - ref32) < 1e-12 * ref32
    # the FP32 positions / weights differ from the FP64 ones by rounding only
    assert abs(ref32 - ref) < 1e-6 * ref
    del torch


def test_axis_tables_and_dispersion_of_the_nodal_cycle():
    p = _params((16, 8, 32), (0.5, 1.0, 0.25), 0.2, (0, 8, 16), (0.0, 0.0, 0.0))
    ctx = context_for(p, cycle=1)
    kc = psatd.nodal_k(p["shape"], [fornberg.k_centered(p["shape"][a], p["dx"][a], p["spectral_order"][a])
                                    for a in range(3)], p["spectral_order"])
    for a in range(3):
        ks, kcd, zt = (np.array(t) for t in ctx.axis_tables(a))
        np.testing.assert_allclose(ks, np.asarray(kc[a], np.float64), rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(kcd, np.asarray(kc[a], np.float64), rtol=1e-14, atol=1e-14)
        assert np.all(zt == 1.0)
    co = psatd.coefficients(p["shape"], p["dx"], p["dt"], p["spectral_order"], nodal=True)
    k = psatd.staggered_k_grid(p["shape"], p["dx"], p["spectral_order"], nodal=True)
    for axis in range(3):
        ref = diagnostics.vacuum_dispersion(co, k, axis, 1.0, p["dt"])
        np.testing.assert_allclose(np.array(ctx.vacuum_dispersion(axis)), ref, rtol=1e-12,
                                   atol=1e-12 * np.max(np.abs(ref)))
