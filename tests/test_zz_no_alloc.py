"""The allocation-free centering entry point (pic_center_to_nodal_static).

It serves callers that may not allocate device memory (their host program owns
all device memory through its own pool, or cannot afford the synchronisation
of cudaMalloc), so it takes no context and keeps its scratch in a static device
array.  Checked through the C ABI against the context-based pic_center_to_nodal,
within the centering tolerance of the other tests, on two calls in a row (the
second call reuses the scratch left by the first).  This file is collected
last so that a failure here stops a -x run only after every other test ran.
"""
import numpy as np
import pytest

from helpers import context_for, to_dev, to_host
from oracle import grid

pytestmark = pytest.mark.gpu


def _params(shape, corder):
    return dict(shape=shape, dx=(1.0, 1.0, 1.0), dt=0.5, shape_order=1, centering_order=corder, variant=0,
                v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0)


@pytest.mark.parametrize("shape,corder", [((16, 8, 32), (8, 4, 16)), ((64, 32, 128), (8, 8, 16)),
                                          ((32, 8, 64), (32, 8, 32))])
def test_static_centering_matches_context_entry_point(shape, corder):
    import torch
    from paper_2106_12919_gb300 import pic
    ctx = context_for(_params(shape, corder))
    for call in range(2):
        rng = np.random.default_rng(100 + call)
        F = [to_dev(rng.normal(size=shape)) for _ in range(6)]
        ref = [torch.empty(ctx.ncell, dtype=torch.float64, device="cuda") for _ in range(6)]
        got = [torch.full((ctx.ncell,), np.nan, dtype=torch.float64, device="cuda") for _ in range(6)]
        ctx.center_to_nodal(F, ref)
        st = pic.center_to_nodal_static(shape, corder, F, got)
        assert st == 0
        torch.cuda.synchronize()
        for c in range(6):
            np.testing.assert_allclose(to_host(got[c]), to_host(ref[c]), rtol=0, atol=1e-14)


def test_static_centering_rejects_grids_beyond_its_scratch():
    # 256 x 128 x 128 = 4,194,304 cells > 2^21: rejected before any launch touches the buffers
    import ctypes
    import torch
    from paper_2106_12919_gb300 import pic
    buf = torch.empty(1, dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * 6)(*([buf.data_ptr()] * 6))
    st = pic.LIB.pic_center_to_nodal_static((ctypes.c_int64 * 3)(256, 128, 128), (ctypes.c_int32 * 3)(8, 8, 8),
                                            ptrs, ptrs, None)
    assert st == -5                              # PIC_ERR_CAPACITY


@pytest.mark.parametrize("shape,corder", [((2, 4, 8), (2, 4, 8)), ((4, 2, 2), (4, 2, 2))])
def test_static_centering_small_grids_match_oracle(shape, corder):
    """Grids of 2 and 4 cells per axis, which pic_init does not take (so there is no context to
    compare with): against the oracle's real-space stencils, two calls in a row."""
    import torch
    from paper_2106_12919_gb300 import pic
    names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
    n = shape[0] * shape[1] * shape[2]
    for call in range(2):
        rng = np.random.default_rng(200 + call)
        F = [rng.normal(size=shape) for _ in range(6)]
        got = [torch.full((n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(6)]
        assert pic.center_to_nodal_static(shape, corder, [to_dev(f) for f in F], got) == 0
        torch.cuda.synchronize()
        for c in range(6):
            ref = grid.center_to_nodal(F[c], names[c], corder)
            np.testing.assert_allclose(to_host(got[c]).reshape(shape), ref, rtol=0, atol=1e-14)


def test_static_centering_rejects_in_place_calls():
    import torch
    from paper_2106_12919_gb300 import pic
    shape = (8, 8, 16)
    F = [torch.zeros(8 * 8 * 16, dtype=torch.float64, device="cuda") for _ in range(6)]
    out = [torch.zeros_like(F[0]) for _ in range(6)]
    out[3] = F[3]
    assert pic.center_to_nodal_static(shape, (4, 4, 4), F, out) == -1     # PIC_ERR_ARG
