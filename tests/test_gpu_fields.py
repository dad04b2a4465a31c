"""GPU parity of the field-side rows: FFT, coefficient tables, centering stencils,
Maxwell solve, diagnostics (libpic through the C ABI vs the oracle)."""
import numpy as np
import pytest

from helpers import TOL, context_for, field_rel_err, to_dev, to_host
from oracle import diagnostics, grid, psatd, step
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 16), (16, 8, 32), (32, 16, 64), (8, 32, 128)]


def _params(shape, variant=0, order=(0, 0, 0), v=(0.0, 0.0, 0.0), corder=(8, 8, 8), dx=(1.0, 0.7, 0.5), dt=0.45):
    return dict(shape=shape, dx=dx, dt=dt, shape_order=1, centering_order=tuple(min(o, s) for o, s in zip(corder, shape)),
                variant=variant, v_gal=v, spectral_order=order, c=1.0, eps0=1.0)


@pytest.mark.parametrize("shape", SHAPES + [(64, 64, 1024), (1024, 8, 16)])
def test_fft_forward_inverse(shape):
    import torch
    ctx = context_for(_params(shape))
    rng = np.random.default_rng(sum(shape))
    f = [rng.normal(size=shape) for _ in range(3)]
    spec = [torch.empty(2 * ctx.nmode, dtype=torch.float64, device="cuda") for _ in range(3)]
    ctx.fft_forward([to_dev(a) for a in f], spec)
    nzh = shape[2] // 2 + 1
    for a, s in zip(f, spec):
        ref = grid.to_spectral(a, "rho", (1.0, 1.0, 1.0))[:, :, :nzh]
        got = to_host(s).reshape(-1, 2)
        got = (got[:, 0] + 1j * got[:, 1]).reshape(shape[0], shape[1], nzh)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-14
    out = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    ctx.fft_inverse(spec, out)
    for a, o in zip(f, out):
        np.testing.assert_allclose(to_host(o).reshape(shape) / a.size, a, atol=1e-13)


COEF_CASES = [
    ((16, 8, 32), 0, (0, 0, 0), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1.0),
    ((16, 8, 32), 0, (8, 8, 16), (0.0, 0.0, 0.0), (0.2, 0.2, 0.04), 0.04),
    ((16, 8, 32), 1, (16, 8, 16), (0.0, 0.0, np.sqrt(1 - 1 / 130.0 ** 2)), (1.0, 1.0, 1.0), 1.0),
    ((16, 16, 64), 2, (16, 16, 16), (0.0, 0.0, np.sqrt(1 - 1e-6)), (0.1, 0.1, 0.02), 0.02),
    ((8, 8, 32), 2, (8, 8, 8), (0.1, -0.2, 0.6), (1.0, 0.8, 0.5), 0.45),
    ((8, 16, 16), 1, (0, 0, 0), (0.0, 0.3, 0.0), (1.0, 1.0, 1.0), 0.9),
]


@pytest.mark.parametrize("case", COEF_CASES)
def test_coefficient_tables(case):
    import torch
    shape, variant, order, v, dx, dt = case
    ctx = context_for(_params(shape, variant, order, v, dx=dx, dt=dt))
    ref = psatd.coefficients(shape, dx, dt, order, v, averaged=variant == 2)
    nzh = shape[2] // 2 + 1
    out = torch.empty(2 * ctx.nmode, dtype=torch.float64, device="cuda")
    for name, r in ref.items():
        ctx.coefficient(name, out)
        g = to_host(out).reshape(-1, 2)
        g = (g[:, 0] + 1j * g[:, 1]).reshape(shape[0], shape[1], nzh)
        r = r[:, :, :nzh]
        err = np.max(np.abs(g - r)) / np.max(np.abs(r))
        assert err < 1e-13, (name, err)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("corder", [(2, 4, 8), (8, 8, 16)])
def test_centering_stencils(shape, corder):
    import torch
    p = _params(shape, corder=corder)
    ctx = context_for(p)
    co = p["centering_order"]
    rng = np.random.default_rng(3)
    F = [rng.normal(size=shape) for _ in range(6)]
    out = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(6)]
    ctx.center_to_nodal([to_dev(f) for f in F], out)
    names = grid.E_NAMES + grid.B_NAMES
    for c in range(6):
        ref = grid.center_to_nodal(F[c], names[c], co)
        np.testing.assert_allclose(to_host(out[c]).reshape(shape), ref, atol=1e-14)
    ctx.center_to_yee([to_dev(f) for f in F[:3]], out[:3])
    for c in range(3):
        ref = grid.center_to_yee(F[c], grid.J_NAMES[c], co)
        np.testing.assert_allclose(to_host(out[c]).reshape(shape), ref, atol=1e-14)


MAXWELL_CASES = [
    ((16, 8, 32), 0, (0, 0, 0), (0.0, 0.0, 0.0)),
    ((16, 16, 32), 0, (16, 16, 16), (0.0, 0.0, 0.0)),
    ((8, 8, 64), 1, (8, 8, 16), (0.0, 0.0, 0.99)),
    ((16, 8, 32), 2, (16, 8, 16), (0.0, 0.0, 0.999)),
    ((8, 16, 16), 2, (8, 8, 8), (0.2, 0.1, -0.3)),
]


@pytest.mark.parametrize("case", MAXWELL_CASES)
def test_maxwell_step(case):
    import torch
    shape, variant, order, v = case
    p = _params(shape, variant, order, v)
    ctx = context_for(p)
    op = step.Params(**p)
    rng = np.random.default_rng(17)
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    J = [rng.normal(size=shape) for _ in range(3)]
    rn, rp = rng.normal(size=shape), rng.normal(size=shape)
    Eo, Bo, avg, _ = step.maxwell_update(op, E, B, J, rn, rp)
    Ed, Bd = [to_dev(a) for a in E], [to_dev(a) for a in B]
    Ea = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    Ba = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(3)]
    ctx.maxwell_step(Ed, Bd, [to_dev(a) for a in J], to_dev(rn), to_dev(rp),
                     Ea if variant == 2 else None, Ba if variant == 2 else None)
    assert field_rel_err([to_host(a).reshape(shape) for a in Ed], Eo) < TOL
    assert field_rel_err([to_host(a).reshape(shape) for a in Bd], Bo) < TOL
    if variant == 2:
        assert field_rel_err([to_host(a).reshape(shape) for a in Ea], avg[0]) < TOL
        assert field_rel_err([to_host(a).reshape(shape) for a in Ba], avg[1]) < TOL


def test_field_energy_and_charge():
    shape = (16, 8, 32)
    p = _params(shape)
    ctx = context_for(p)
    rng = np.random.default_rng(2)
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    Ed, Bd = [to_dev(a) for a in E], [to_dev(a) for a in B]
    W = ctx.field_energy(Ed, Bd)
    assert abs(W - diagnostics.field_energy(E, B, p["dx"])) < 1e-13 * W
    # boxes: ragged z (scalar path), z a multiple of 4 (vector path), whole y-z planes (contiguous)
    for lo, hi in (((2, 1, 5), (9, 7, 30)), ((3, 2, 4), (16, 5, 28)), ((5, 0, 0), (11, 8, 32))):
        Wb = ctx.field_energy(Ed, Bd, lo, hi)
        assert abs(Wb - diagnostics.field_energy(E, B, p["dx"], box_lo=lo, box_hi=hi)) < 1e-13 * Wb
    # FP32 form: FP64 sums of the FP32 data
    from paper_2106_12919_gb300 import pic
    import torch
    c32 = context_for(p, precision=pic.PIC_FP32)
    E32 = [a.astype(np.float32) for a in E]
    B32 = [a.astype(np.float32) for a in B]
    d32 = lambda a: torch.from_numpy(a).cuda()
    # values spread over twelve decades: the FP32 partial sums must carry the small terms
    E32[0] *= np.exp(rng.uniform(-14, 14, size=shape)).astype(np.float32)
    for lo, hi in ((None, None), ((2, 1, 5), (9, 7, 30)), ((5, 0, 0), (11, 8, 32))):
        Wf = c32.field_energy32([d32(a) for a in E32], [d32(a) for a in B32], lo, hi)
        ref = diagnostics.field_energy([a.astype(np.float64) for a in E32], [a.astype(np.float64) for a in B32],
                                       p["dx"], box_lo=lo, box_hi=hi)
        assert abs(Wf - ref) < 1e-13 * ref
    rho = rng.normal(size=shape)
    q = ctx.total_charge(to_dev(rho))
    assert abs(q - np.sum(rho) * np.prod(p["dx"])) < 1e-12 * np.sum(np.abs(rho))
