"""GPU checks of the reverse mode (pic_adjoint_step and the ProbeEnergy autograd.Function):
one adjoint step against the oracle's adjoint step, gradients against the oracle's full
reverse pass, and gradients against central finite differences of the GPU forward
(eps = 1e-6, agreement within 1e-6 relative) on the differentiable probe workload."""
import numpy as np
import pytest

from helpers import context_for, field_rel_err, species_to_dev, to_dev, to_host
from oracle import adjoint as oadj
from oracle import step
from paper_2106_12919_gb300 import workloads

pytestmark = pytest.mark.gpu


def _adj_dev(d):
    return {k: to_dev(v) for k, v in d.items()}


@pytest.mark.parametrize("name,kw,order", [("seed_wave", dict(shape=(16, 16, 16), ppc=2), 1),
                                           ("seed_wave", dict(shape=(16, 16, 32), ppc=1), 3),
                                           ("galilean_drift", dict(shape=(16, 16, 32), ppc=1), 2)])
def test_adjoint_step_matches_oracle(name, kw, order):
    import torch
    w = workloads.WORKLOADS[name](**kw)
    prm = dict(w["params"])
    prm["shape_order"] = order
    p = step.Params(**prm)
    shape = p.shape
    ctx = context_for(prm, sort_interval=0)
    st = {"E": w["E"], "B": w["B"], "species": w["species"]}
    st["rho"] = step.initial_rho(p, st["species"])
    rng = np.random.default_rng(4)
    adj = {"E": [rng.normal(size=shape) for _ in range(3)], "B": [rng.normal(size=shape) for _ in range(3)],
           "rho": rng.normal(size=shape),
           "species": [{k: rng.normal(size=s["x"].size) for k in ("x", "y", "z", "ux", "uy", "uz")}
                       for s in w["species"]]}
    ref = oadj.adjoint_step(p, st, adj)
    Ed, Bd = [to_dev(a) for a in w["E"]], [to_dev(a) for a in w["B"]]
    sp = species_to_dev(w["species"], with_id=False)
    Eb, Bb = [to_dev(a) for a in adj["E"]], [to_dev(a) for a in adj["B"]]
    rb = to_dev(adj["rho"])
    spb = [_adj_dev(d) for d in adj["species"]]
    ctx.adjoint_step(Ed, Bd, sp, Eb, Bb, rb, spb)
    ctx.sync()
    g = lambda ts: [to_host(t).reshape(shape) for t in ts]
    assert field_rel_err(g(Eb), ref["E"]) < 1e-11
    assert field_rel_err(g(Bb), ref["B"]) < 1e-11
    assert field_rel_err(g([rb]), [ref["rho"]]) < 1e-11
    for gs, rs in zip(spb, ref["species"]):
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            assert np.linalg.norm(to_host(gs[k]) - rs[k]) < 1e-11 * np.linalg.norm(rs[k]), k


def _probe_run(shape, ppc, steps, K, amplitude=0.01, order=1):
    import torch
    from paper_2106_12919_gb300 import adjoint as gadj
    w = workloads.seed_wave(shape=shape, ppc=ppc, amplitude=amplitude)
    p = dict(w["params"])
    p["shape_order"] = order
    w["params"] = p
    ctx = context_for(p, sort_interval=0)
    (sp,) = species_to_dev(w["species"], with_id=False)
    lo, hi = w["probe"]
    run = gadj.Rollout(ctx, [sp], steps, lo, hi, checkpoint=K)
    profile = to_dev(w["E"][0] / amplitude)
    E0 = torch.stack([to_dev(a) for a in w["E"]])
    B0 = torch.stack([to_dev(a) for a in w["B"]])
    return w, run, sp, profile, E0, B0


def _forward_cells(run, sp, E0, B0, A, profile, du=None, margins=False):
    """Probe loss of one forward run and the cell index of every particle at every step
    (state positions and the midpoints that carry the J deposit); with margins=True also each
    particle's smallest distance (in cells) to a cell face over those positions."""
    import torch
    from paper_2106_12919_gb300 import pic
    ctx = run.ctx
    E = [E0[a].clone() for a in range(3)]
    E[0] = A * profile
    B = [B0[a].clone() for a in range(3)]
    s = pic.Species(sp.x.clone(), sp.y.clone(), sp.z.clone(), sp.ux.clone(), sp.uy.clone(), sp.uz.clone(), sp.w,
                    sp.q, sp.m)
    if du is not None:
        s.ux += du[0]
        s.uy += du[1]
        s.uz += du[2]
    rho = torch.empty_like(E[0])
    ctx.deposit_rho([s], rho)
    dx = ctx.dx
    L = [ctx.shape[a] * dx[a] for a in range(3)]
    cells = []
    near = torch.full_like(s.x, 1.0)
    for _ in range(run.nsteps):
        x0 = [s.x.clone(), s.y.clone(), s.z.clone()]
        J = [torch.empty_like(rho) for _ in range(3)]
        ctx.step(E, B, J, rho, [s], 1)
        x1 = [s.x, s.y, s.z]
        for a in range(3):
            d = torch.remainder(x1[a] - x0[a] + 0.5 * L[a], L[a]) - 0.5 * L[a]    # unwrapped displacement
            mid = torch.remainder(x0[a] + 0.5 * d, L[a])
            cells.append(torch.floor(x1[a] / dx[a]).to(torch.int32))
            cells.append(torch.floor(mid / dx[a]).to(torch.int32))
            if margins:
                for v in (x1[a] / dx[a], mid / dx[a]):
                    f = v - torch.floor(v)
                    near = torch.minimum(near, torch.minimum(f, 1.0 - f))
    if margins:
        return ctx.field_energy(E, B, run.lo, run.hi), cells, near
    return ctx.field_energy(E, B, run.lo, run.hi), cells


def _fd(run, sp, E0, B0, A, profile, grad, eps, du=None, repeats=4, kinks=True):
    """Central difference with the smallest tried eps whose +/- runs cross no cell face.

    The FP64 deposits are atomic, so their summation order (and the loss, at ~1e-16 of it per
    step, amplified by the plasma) varies from run to run; the difference is averaged over
    `repeats` independent +/- pairs and returned with its standard error."""
    for _ in range(6):
        dp = None if du is None else [eps * d for d in du]
        dm = None if du is None else [-eps * d for d in du]
        vals = []
        for _ in range(repeats):
            Lp, cp = _forward_cells(run, sp, E0, B0, A + (0 if du is not None else eps), profile, dp)
            Lm, cm = _forward_cells(run, sp, E0, B0, A - (0 if du is not None else eps), profile, dm)
            if kinks and sum(int((a != b).sum()) for a, b in zip(cp, cm)):
                break
            vals.append((Lp - Lm) / (2 * eps))
        if len(vals) == repeats:
            v = np.array(vals)
            return float(v.mean()), eps, float(v.std(ddof=1) / np.sqrt(repeats))
        eps /= 10.0
    raise AssertionError("no crossing-free finite-difference step found")


@pytest.mark.parametrize("shape,ppc,steps,K,order,bound", [
    ((32, 32, 32), 2, 12, 5, 3, None), ((32, 32, 32), 2, 12, 5, 1, None),
    # the full probe grid and particle count (64^3, 1M particles): cubic (C2, no kinks) at 1e-6;
    # CIC, whose kinks force eps towards the rounding of the loss, at the bound it can resolve
    ((64, 64, 64), 4, 12, 5, 3, None), ((64, 64, 64), 4, 50, 10, 3, None),
    ((64, 64, 64), 4, 12, 5, 1, 1e-4), ((64, 64, 64), 4, 50, 10, 1, 1e-3)])
def test_gradient_matches_central_differences(shape, ppc, steps, K, order, bound):
    """Central differences with eps = 1e-6 relative to the parameter (A, or |u0| for unit
    directions in momentum space), each the mean of four independent +/- pairs: the FP64
    deposits are atomic and their summation order varies from run to run, so the bound is
    1e-6 relative plus four standard errors of that mean (a momentum direction's error relative
    to the larger of its derivative and the typical one, ||g|| / sqrt(3n)).  The cubic shape is C2 and eps stays
    at 1e-6.  The CIC shape is only piecewise linear: eps is reduced by tens while a +/- run
    crosses a cell face, and momentum directions are drawn on the particles that stay 1e-4 cells
    away from every face (the field response still moves the others).  On 32^3 that keeps 1e-6;
    with the full 1M particles crossings drive eps to 1e-7..1e-9, where the difference of the two
    losses nears their rounding and a thermal plasma's amplified deposit noise (~1e-12 of the
    loss after 50 steps): those CIC cases are held to 1e-4 (12 steps) and 1e-3 (50 steps), and
    the 1e-10 agreement with the oracle's own reverse pass checks the CIC adjoint exactly."""
    import torch
    from paper_2106_12919_gb300 import adjoint as gadj
    amp = 0.01
    w, run, sp, profile, E0, B0 = _probe_run(shape, ppc, steps, K, amp, order)
    A = torch.tensor(amp, dtype=torch.float64, device="cuda", requires_grad=True)
    ux = sp.ux.clone().requires_grad_(True)
    uy = sp.uy.clone().requires_grad_(True)
    uz = sp.uz.clone().requires_grad_(True)
    Bz = torch.zeros_like(profile)
    E = torch.stack([A * profile, Bz, Bz])
    loss = gadj.ProbeEnergy.apply(E, B0, ux, uy, uz, run)
    loss.backward()
    gA = float(A.grad)
    gu = [ux.grad, uy.grad, uz.grad]
    kinks = order == 1
    fdA, epsA, seA = _fd(run, sp, E0, B0, amp, profile, gA, 1e-6 * amp, kinks=kinks)
    # 1e-6 plus four standard errors of the averaged difference (the run-to-run noise)
    tolA = bound if bound else 1e-6 + 4 * seA / abs(fdA)
    print("\ndL/dA adjoint %.12e  FD %.12e (eps %.1e, s.e. %.1e)  rel %.2e  bound %.1e" %
          (gA, fdA, epsA, seA / abs(fdA), abs(gA - fdA) / abs(fdA), tolA))
    assert abs(gA - fdA) < tolA * abs(fdA)
    g = torch.Generator(device="cuda").manual_seed(7)
    n = sp.n
    unorm = float(torch.sqrt(torch.sum(sp.ux ** 2 + sp.uy ** 2 + sp.uz ** 2)))
    # momentum directions on the particles that stay 1e-4 cells from every face along the run:
    # a relative eps of 1e-6 moves a trajectory by ~1e-6 cells, so the +/- runs cross no face
    # and the difference keeps ~10 digits above the rounding of the loss
    _, _, near = _forward_cells(run, sp, E0, B0, amp, profile, margins=True)
    keep = (near > 1e-4).to(torch.float64)
    print("momentum directions on %.1f%% of the particles" % (100.0 * float(keep.mean())))
    # the typical size of g . d for a random unit d on that support: ||g|| / sqrt(components)
    gnorm = float(torch.sqrt(sum(torch.sum((gu[a] * keep) ** 2) for a in range(3))))
    typical = gnorm / np.sqrt(3.0 * float(keep.sum()))
    for trial in range(8 if shape[0] == 64 else 3):
        d = torch.randn(3, n, dtype=torch.float64, device="cuda", generator=g) * keep
        d /= torch.linalg.norm(d)
        ad = float(sum(torch.dot(gu[a], d[a]) for a in range(3)))
        fd, eps, se = _fd(run, sp, E0, B0, amp, profile, ad, 1e-6 * unorm, du=[d[0], d[1], d[2]], kinks=kinks)
        # relative to the larger of |fd| and the typical directional derivative, so that a
        # direction nearly orthogonal to the gradient does not turn rounding into a relative error
        scale = max(abs(fd), typical)
        tol = bound if bound else 1e-6 + 4 * se / scale
        rel = abs(ad - fd) / scale
        print("direction %d: adjoint %.12e  FD %.12e (eps %.1e, s.e. %.1e)  rel %.2e  bound %.1e" %
              (trial, ad, fd, eps, se / abs(fd), rel, tol))
        assert rel < tol


def test_gradient_matches_oracle_reverse_pass():
    import torch
    from paper_2106_12919_gb300 import adjoint as gadj
    amp = 0.05
    w, run, sp, profile, E0, B0 = _probe_run((16, 16, 16), 2, 6, 4, amp)
    ux = sp.ux.clone().requires_grad_(True)
    uy = sp.uy.clone().requires_grad_(True)
    uz = sp.uz.clone().requires_grad_(True)
    Er = E0.clone().requires_grad_(True)
    loss = gadj.ProbeEnergy.apply(Er, B0, ux, uy, uz, run)
    loss.backward()
    p = step.Params(**w["params"])
    st = {"E": w["E"], "B": w["B"], "species": w["species"]}
    st["rho"] = step.initial_rho(p, st["species"])
    L, adj = oadj.loss_and_gradient(p, st, 6, *w["probe"], checkpoint=4)
    assert abs(float(loss.detach()) - L) < 1e-12 * L
    for k, t in (("ux", ux), ("uy", uy), ("uz", uz)):
        r = adj["species"][0][k]
        assert np.linalg.norm(to_host(t.grad) - r) < 1e-10 * np.linalg.norm(r), k
    gE = to_host(Er.grad)
    assert field_rel_err([gE[a].reshape(p.shape) for a in range(3)], adj["E"]) < 1e-10
