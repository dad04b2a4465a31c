"""The FP32 form against the plain FP64 form on the same GPU, at the full workload sizes.

The FP64 form is held to the oracle at 1e-12 per step (test_gpu_step.py, test_gpu_fullsize.py), so
here it stands in for the FP64 reference where the oracle would take hours:

* the laser-wakefield box (128 x 128 x 512, 16.8M particles, standard PSATD, cubic) and the
  beam-driven box (256 x 256 x 1024, 68.1M particles, averaged Galilean PSATD, cubic), 100 steps
  in both forms: every E and B component within 1e-5 (Eq. L2_norm_error, Sec. 5.2, per
  component), and J, rho and each momentum component within 1e-5 as well.  A component below
  1 % of its field's largest one (B_z of the axisymmetric beam wake: a residue of the cancelling
  curl of the large transverse E) carries the FP32 rounding of the large components, so it is
  measured against its field's largest component instead of its own norm;
* the drifting pair plasma (64 x 64 x 256, 4.2M particles, Galilean PSATD, quadratic), whose
  field energy W(t) the workload tracks over 500 steps: the thermal noise makes the particle
  trajectories chaotic, so the two forms are compared on W(t), a sum over a million cells, which
  two microscopically different runs share to its statistical fluctuation (~1e-3); it is held
  to 1e-2 of W(t) at every step.
"""
import numpy as np
import pytest

from helpers import context_for, periodic_pos_err, to_host
from paper_2106_12919_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def component_errors(gpu, ref):
    """||a_c - b_c|| / ||b_c|| per component (Eq. L2_norm_error); a component below 1 % of its
    field's largest one is measured against that one's norm instead."""
    norms = [float(np.linalg.norm(r)) for r in ref]
    big = max(norms)
    return [float(np.linalg.norm(a - r)) / (nr if nr >= 1e-2 * big else max(big, 1e-300))
            for a, r, nr in zip(gpu, ref, norms)]


def _run(w, form, nsteps):
    """nsteps of one form on the workload; host results in the original particle order."""
    import torch
    from paper_2106_12919_gb300 import pic
    p = w["params"]
    fp32 = form == "fp32"
    ctx = context_for(p, precision=pic.PIC_FP32 if fp32 else pic.PIC_FP64)
    dt = torch.float32 if fp32 else torch.float64
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt).reshape(-1)
    E, B = [dev(a) for a in w["E"]], [dev(a) for a in w["B"]]
    J = [torch.empty(ctx.ncell, dtype=dt, device="cuda") for _ in range(3)]
    rho = torch.empty(ctx.ncell, dtype=dt, device="cuda")
    sp = []
    for s in w["species"]:
        ids = torch.arange(s["x"].size, dtype=torch.int64, device="cuda")
        if fp32:
            sp.append(pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                                   s["q"], s["m"], id=ids))
        else:
            d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            sp.append(pic.Species(d(s["x"]), d(s["y"]), d(s["z"]), d(s["ux"]), d(s["uy"]), d(s["uz"]), d(s["w"]),
                                  s["q"], s["m"], id=ids))
    (ctx.deposit_rho32 if fp32 else ctx.deposit_rho)(sp, rho)
    (ctx.step32 if fp32 else ctx.step)(E, B, J, rho, sp, nsteps)
    ctx.sync()
    shape = p["shape"]
    h = lambda t: to_host(t).astype(np.float64).reshape(shape)
    out = {"E": [h(t) for t in E], "B": [h(t) for t in B], "J": [h(t) for t in J], "rho": [h(rho)], "species": []}
    for s in sp:
        s64 = ctx.species32_to_species(s) if fp32 else s
        ctx.sync()
        ids = to_host(s64.id)
        d = {}
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            v = np.empty(s.n)
            v[ids] = to_host(getattr(s64, k))
            d[k] = v
        out["species"].append(d)
    ctx.close()
    del E, B, J, rho, sp
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("name", ["laser_wakefield", "beam_wakefield"])
def test_fp32_form_within_1e5_of_fp64_form_after_100_steps(name):
    w = workloads.WORKLOADS[name]()
    p = w["params"]
    r64 = _run(w, "fp64", 100)
    r32 = _run(w, "fp32", 100)
    errs = {k: component_errors(r32[k], r64[k]) for k in ("E", "B", "J", "rho")}
    mom = {}
    for k in ("ux", "uy", "uz"):
        a = np.concatenate([s[k] for s in r32["species"]])
        b = np.concatenate([s[k] for s in r64["species"]])
        mom[k] = float(np.linalg.norm(a - b)) / max(float(np.linalg.norm(b)), 1e-300)
    pos = {}
    for ax, k in enumerate(("x", "y", "z")):
        L = p["shape"][ax] * p["dx"][ax]
        d = np.concatenate([periodic_pos_err(s32[k], s64[k], L) for s32, s64 in zip(r32["species"], r64["species"])])
        pos[k] = float(np.max(d)) / p["dx"][ax]
    share = {k: [float(np.linalg.norm(r)) / max(float(np.linalg.norm(x)) for x in r64[k]) for r in r64[k]]
             for k in ("E", "B", "J")}
    print("\n%s, FP32 vs FP64 form after 100 steps: per component %s\n component norms / field's largest %s"
          "\n momenta %s\n max position error (cells) %s" % (name, errs, share, mom, pos))
    for k in ("E", "B", "J", "rho"):
        assert max(errs[k]) < 1e-5, (k, errs[k])
    assert max(mom.values()) < 1e-5, mom
    assert max(pos.values()) < 1e-3, pos


def test_galilean_drift_field_energy_history_fp32_vs_fp64():
    import torch
    from paper_2106_12919_gb300 import pic
    w = workloads.galilean_drift()
    p = w["params"]
    nsteps = w["steps"]
    hist = {}
    for form in ("fp64", "fp32"):
        fp32 = form == "fp32"
        ctx = context_for(p, precision=pic.PIC_FP32 if fp32 else pic.PIC_FP64)
        dt = torch.float32 if fp32 else torch.float64
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt).reshape(-1)
        E, B = [dev(a) for a in w["E"]], [dev(a) for a in w["B"]]
        rho = torch.empty(ctx.ncell, dtype=dt, device="cuda")
        if fp32:
            sp = [pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                               s["q"], s["m"]) for s in w["species"]]
        else:
            d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            sp = [pic.Species(d(s["x"]), d(s["y"]), d(s["z"]), d(s["ux"]), d(s["uy"]), d(s["uz"]), d(s["w"]),
                              s["q"], s["m"]) for s in w["species"]]
        (ctx.deposit_rho32 if fp32 else ctx.deposit_rho)(sp, rho)
        step = ctx.step32 if fp32 else ctx.step
        energy = ctx.field_energy32 if fp32 else ctx.field_energy
        W = []
        for _ in range(nsteps):
            step(E, B, None, rho, sp, 1)
            W.append(energy(E, B))
        hist[form] = np.array(W)
        ctx.close()
        del E, B, rho, sp
        torch.cuda.empty_cache()
    W64, W32 = hist["fp64"], hist["fp32"]
    rel = np.abs(W32 - W64) / W64
    marks = [0, 9, 49, 99, 199, 299, 399, 499]
    print("\ngalilean_drift W(t): " + ", ".join("step %d: W64 %.4e W32 %.4e rel %.1e" % (k + 1, W64[k], W32[k], rel[k])
                                                  for k in marks))
    assert np.all(np.isfinite(W32)) and np.all(W64 > 0)
    assert float(np.max(rel)) < 1e-2, float(np.max(rel))
