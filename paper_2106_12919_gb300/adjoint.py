"""Reverse-mode differentiation of the hybrid PIC step behind torch.autograd.

:class:`ProbeEnergy` is a ``torch.autograd.Function`` whose forward runs
``nsteps`` FP64 hybrid PIC steps through ``pic_step`` and returns the field
energy of a probe box (``pic_field_energy``); its backward runs the adjoint
chain through ``pic_adjoint_step``.  Forward states are checkpointed every
``checkpoint`` steps; backward recomputes each segment forward (one
``pic_step`` per step) and reverses it.  Everything stays on the device; this
module only marshals tensors and orders the library calls.

The context must be FP64, standard or Galilean, and created with
``sort_interval = 0`` so that particle order stays fixed between the forward
and the adjoint passes.
"""
import torch

from . import pic


class Rollout:
    """Static part of a differentiable run: context, positions and weights, steps, probe box."""

    def __init__(self, ctx, species, nsteps, box_lo, box_hi, checkpoint=10):
        if ctx.precision != pic.PIC_FP64:
            raise ValueError("the differentiable form is FP64")
        if ctx.sort_interval != 0:
            raise ValueError("create the context with sort_interval=0: particle order must stay fixed")
        if len(species) != 1:
            raise ValueError("ProbeEnergy differentiates one species")
        self.ctx, self.species, self.nsteps = ctx, species, int(nsteps)
        self.lo, self.hi, self.K = tuple(box_lo), tuple(box_hi), int(checkpoint)


def _clone_state(E, B, rho, sp):
    return ([t.clone() for t in E], [t.clone() for t in B], rho.clone(),
            [pic.Species(s.x.clone(), s.y.clone(), s.z.clone(), s.ux.clone(), s.uy.clone(), s.uz.clone(), s.w,
                         s.q, s.m) for s in sp])


class ProbeEnergy(torch.autograd.Function):
    """loss = W over the probe box after ``run.nsteps`` steps, as a function of the initial
    Yee fields E, B (tensors of shape (3, ncell)) and the initial momenta ux, uy, uz of each
    species (lists, one tensor per species)."""

    @staticmethod
    def forward(fctx, E, B, ux, uy, uz, run):
        ctx = run.ctx
        sp0 = [pic.Species(s.x, s.y, s.z, a, b, c_, s.w, s.q, s.m) for s, a, b, c_ in
               zip(run.species, [ux], [uy], [uz])]
        Ec, Bc = [E[a].clone() for a in range(3)], [B[a].clone() for a in range(3)]
        rho = torch.empty_like(E[0])
        sp = _clone_state(Ec, Bc, rho, sp0)[3]
        ctx.deposit_rho(sp, rho)
        ckpt = {}
        for n in range(run.nsteps):
            if n % run.K == 0:
                ckpt[n] = _clone_state(Ec, Bc, rho, sp)
            J = [torch.empty_like(rho) for _ in range(3)]
            ctx.step(Ec, Bc, J, rho, sp, 1)
        loss = ctx.field_energy(Ec, Bc, run.lo, run.hi)
        fctx.run = run
        fctx.ckpt = ckpt
        fctx.final = (Ec, Bc)
        return torch.tensor(loss, dtype=torch.float64, device=E.device)

    @staticmethod
    def backward(fctx, gout):
        run = fctx.run
        ctx = run.ctx
        Ec, Bc = fctx.final
        # the seed g dW/dE, g dW/dB of the probe box (pic_field_energy_adjoint); every adjoint
        # below is linear in it, so the returned gradients already carry the factor g
        Eb = [torch.empty_like(Ec[0]) for _ in range(3)]
        Bb = [torch.empty_like(Ec[0]) for _ in range(3)]
        ctx.field_energy_adjoint(Ec, Bc, run.lo, run.hi, float(gout), Eb, Bb)
        rhob = torch.zeros_like(Ec[0])
        spb = [{k: torch.zeros_like(s.x) for k in ("x", "y", "z", "ux", "uy", "uz")} for s in run.species]
        for s0 in sorted(fctx.ckpt, reverse=True):
            s1 = min(s0 + run.K, run.nsteps)
            E, B, rho, sp = _clone_state(*fctx.ckpt[s0])
            states = []
            for n in range(s0, s1):
                states.append(_clone_state(E, B, rho, sp))
                if n < s1 - 1:
                    J = [torch.empty_like(rho) for _ in range(3)]
                    ctx.step(E, B, J, rho, sp, 1)
            for n in range(s1 - 1, s0 - 1, -1):
                Es, Bs, _, sps = states[n - s0]
                ctx.adjoint_step(Es, Bs, sps, Eb, Bb, rhob, spb)
        return torch.stack(Eb), torch.stack(Bb), spb[0]["ux"], spb[0]["uy"], spb[0]["uz"], None
