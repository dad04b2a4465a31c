"""GPU checks of the representation conversions and of the probe-energy adjoint seed, all
through the C ABI, against the oracle.

pic_species32_from_species must reproduce the oracle's (cell, FP32 offset) split bit for bit
(integer cells and the single FP32 rounding of the offset), pic_species32_to_species its FP64 join,
and pic_field_energy_adjoint the oracle's dW/dE, dW/dB of the probe box (Sec. 2 (iii))."""
import numpy as np
import pytest

from helpers import context_for, to_host
from oracle import adjoint, particles, step

pytestmark = pytest.mark.gpu


def _params(shape, dx, **kw):
    p = dict(shape=shape, dx=dx, dt=0.5 * min(dx), shape_order=3, centering_order=(4, 4, 8), variant=0,
             v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)
    p.update(kw)
    return p


def _positions(rng, shape, dx, n):
    """Uniform positions plus the hard cases: cell faces, the last double below each face and
    below the box end, offsets that round up to 1 in FP32, and 0."""
    L = [shape[a] * dx[a] for a in range(3)]
    pos = [rng.uniform(0.0, L[a], n) for a in range(3)]
    for a in range(3):
        faces = np.arange(shape[a]) * dx[a]
        below = np.nextafter(faces[1:], 0.0)
        near = (np.arange(shape[a]) + 1 - 2.0 ** -30) * dx[a]
        extra = np.concatenate([faces, below, near[near < L[a]], [0.0, np.nextafter(L[a], 0.0)]])
        pos[a][:extra.size] = extra
    return pos


@pytest.mark.parametrize("shape,dx", [((16, 8, 32), (0.2, 0.2, 0.04)), ((8, 64, 16), (1.0, 0.1, 0.3)),
                                      ((128, 128, 512), (0.2, 0.2, 0.04))])
def test_species32_split_and_join_bit_exact(shape, dx):
    import torch
    from paper_2106_12919_gb300 import pic
    ctx = context_for(_params(shape, dx), precision=pic.PIC_FP32)
    rng = np.random.default_rng(3)
    n = 200003                                   # ragged: not a multiple of the block size
    x, y, z = _positions(rng, shape, dx, n)
    u = [rng.normal(0.0, 3.0, n) for _ in range(3)]
    w = rng.uniform(0.1, 2.0, n)
    ids = torch.arange(n, dtype=torch.int64, device="cuda") * 7
    sp = pic.Species32.from_positions(ctx, x, y, z, *u, w, -1.0, 1.0, id=ids)
    ctx.sync()
    ref = [particles.cell_offset_split(v, dx[a], shape[a]) for a, v in enumerate((x, y, z))]
    cell = particles.linear_cell(ref[0][0], ref[1][0], ref[2][0], shape)
    np.testing.assert_array_equal(to_host(sp.cell).astype(np.int64), cell)
    for a, k in enumerate(("fx", "fy", "fz")):
        got = to_host(getattr(sp, k))
        assert got.dtype == np.float32
        np.testing.assert_array_equal(got.view(np.uint32), ref[a][1].view(np.uint32))
    for k, v in zip(("ux", "uy", "uz", "w"), u + [w]):
        np.testing.assert_array_equal(to_host(getattr(sp, k)).view(np.uint32), v.astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(to_host(sp.id), np.arange(n) * 7)
    # some offsets did round up to 1 and moved to the next cell
    base = np.floor(x * (1.0 / dx[0])).astype(np.int64) % shape[0]
    assert np.any(ref[0][0] != base)
    # join: x = (i + f) dx in FP64, u and w widened
    s64 = ctx.species32_to_species(sp)
    ctx.sync()
    for a, k in enumerate(("x", "y", "z")):
        want = particles.cell_offset_join(ref[a][0], ref[a][1], dx[a])
        np.testing.assert_array_equal(to_host(getattr(s64, k)), want)
    for k, v in zip(("ux", "uy", "uz", "w"), u + [w]):
        np.testing.assert_array_equal(to_host(getattr(s64, k)), v.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(to_host(s64.id), np.arange(n) * 7)


def test_species32_conversion_empty_and_errors():
    import torch
    from paper_2106_12919_gb300 import pic
    ctx = context_for(_params((8, 8, 16), (1.0, 1.0, 1.0)), precision=pic.PIC_FP32)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    sp = pic.Species32.from_positions(ctx, e, e, e, e, e, e, e, -1.0, 1.0)
    assert sp.n == 0
    ctx.sync()
    # counts that differ, and an id on one side only
    s64 = pic.Species(*[torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(7)], -1.0, 1.0)
    s32 = pic.Species32(torch.zeros(3, dtype=torch.int32, device="cuda"),
                        *[torch.zeros(3, dtype=torch.float32, device="cuda") for _ in range(7)], -1.0, 1.0)
    with pytest.raises(pic.PicError):
        ctx._check(pic.LIB.pic_species32_from_species(ctx.h, pic.ctypes.byref(s64.c_struct()),
                                                      pic.ctypes.byref(s32.c_struct())))
    s64.id = torch.zeros(4, dtype=torch.int64, device="cuda")
    s32 = ctx.species32_from_species(pic.Species(*s64.arrays(), -1.0, 1.0))
    with pytest.raises(pic.PicError):
        ctx._check(pic.LIB.pic_species32_from_species(ctx.h, pic.ctypes.byref(s64.c_struct()),
                                                      pic.ctypes.byref(s32.c_struct())))


@pytest.mark.parametrize("box,c,eps0,scale", [(((3, 2, 5), (11, 7, 30)), 1.0, 1.0, 1.0),
                                              (((0, 0, 0), (16, 8, 32)), 2.0, 0.5, -3.25),
                                              (None, 1.5, 3.0, 0.125)])
def test_field_energy_adjoint_matches_oracle(box, c, eps0, scale):
    import torch
    shape, dx = (16, 8, 32), (0.5, 1.0, 0.25)
    p = _params(shape, dx, c=c, eps0=eps0)
    ctx = context_for(p)
    rng = np.random.default_rng(8)
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    lo, hi = box if box is not None else ((0, 0, 0), shape)
    Eb = [torch.full((ctx.ncell,), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
    Bb = [torch.full((ctx.ncell,), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().reshape(-1)
    ctx.field_energy_adjoint([dev(a) for a in E], [dev(a) for a in B], box[0] if box else None,
                             box[1] if box else None, scale, Eb, Bb)
    ctx.sync()
    rE, rB = adjoint.probe_energy_bar(step.Params(**p), E, B, lo, hi)
    for g, r in zip(Eb + Bb, rE + rB):
        g = to_host(g).reshape(shape)
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - scale * r)) <= 1e-15 * np.max(np.abs(scale * r))
        assert np.all(g[r == 0] == 0)
