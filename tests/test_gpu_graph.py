"""pic.StepGraph: a pic_step / pic_step32 call captured into a CUDA graph and replayed gives the
same result as the direct call on the same inputs (every decision of the step is on the device)."""
import numpy as np
import pytest

from helpers import context_for, field_rel_err, species_to_dev, to_dev, to_host
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
def test_graph_replay_matches_direct_call(fp32):
    import torch
    from paper_2106_12919_gb300 import pic
    w = workloads.laser_wakefield(shape=(16, 16, 64), ppc=2)
    p = w["params"]
    shape, dx = p["shape"], p["dx"]
    stream = torch.cuda.Stream()
    ctx = context_for(p, sort_interval=5, stream=stream,
                      **({"precision": pic.PIC_FP32} if fp32 else {}))
    dt = np.float32 if fp32 else np.float64
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()

    def fresh():
        if fp32:
            sp = [pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                               s["q"], s["m"]) for s in w["species"]]
        else:
            sp = species_to_dev(w["species"], with_id=False)
        return [dev(a) for a in w["E"]], [dev(a) for a in w["B"]], torch.zeros(ctx.ncell, dtype=dev(w["E"][0]).dtype,
                                                                              device="cuda"), sp

    with torch.cuda.stream(stream):
        E, B, rho, sp = fresh()
        (ctx.deposit_rho32 if fp32 else ctx.deposit_rho)(sp, rho)
    ctx.sync()
    # inputs of the comparison, kept on the host
    init = [to_host(t).copy() for t in E + B + [rho]] + [to_host(a).copy() for s in sp for a in s.arrays()]
    cap = ctx.capture_step32 if fp32 else ctx.capture_step
    J = [torch.empty(ctx.ncell, dtype=rho.dtype, device="cuda") for _ in range(3)]
    g = cap(E, B, J, rho, sp, 3)
    outs = []
    for replay in (False, True):
        arrs = E + B + [rho] + [a for s in sp for a in s.arrays()]
        for t, h in zip(arrs, init):
            t.copy_(torch.from_numpy(h))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            if replay:
                g.replay()
            else:
                (ctx.step32 if fp32 else ctx.step)(E, B, J, rho, sp, 3)
        torch.cuda.synchronize()
        outs.append([to_host(t).astype(np.float64) for t in E + B + J + [rho]])
    tol = 1e-6 if fp32 else 1e-13
    assert field_rel_err(outs[1][:6], outs[0][:6]) < tol
    assert field_rel_err(outs[1][6:9], outs[0][6:9]) < tol
    assert field_rel_err([outs[1][9]], [outs[0][9]]) < tol
