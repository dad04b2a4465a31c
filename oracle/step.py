"""The hybrid PSATD PIC cycle (Sec. 2, the "hybrid PSATD PIC cycle" diagram).

Test infrastructure only (see oracle/__init__.py).

One step, in the paper's order:
  1. finite-order centering of E, B from the Yee grid to the nodal grid (Sec. 3);
  2. gather E, B from the nodal grid, push particles (x^n, u^{n-1/2} -> x^{n+1}, u^{n+1/2});
  3. deposit J^{n+1/2} and rho^{n+1} on the nodal grid;
  4. finite-order centering of J from the nodal grid to the Yee grid (rho stays nodal);
  5. solve Maxwell's equations on the Yee grid in Fourier space (Sec. 4): forward
     transforms, PSATD update, inverse transforms.

Comparison cycles (Sec. 2, the "standard" PSATD PIC cycle): NODAL: every quantity on the
nodes, the centered modified wave numbers [k]_c in the solver, no centering; STAGGERED: the
Yee-grid solver of the hybrid cycle, with E, B gathered from and J deposited at their own Yee
positions (rho nodal), no centering.

Hybrid FDTD cycle (the FDTD adaptation the conclusions of Sec. 6 point to): the hybrid cycle with
step 5 replaced by the Yee finite-difference update of oracle/fdtd.py (order 2m per axis from the
spectral-order argument, 0 meaning Yee's order 2); rho^n, rho^{n+1} are not used by the solver.

Averaged Galilean variant (Sec. 4.4): the Yee state E, B evolves with the
Galilean update; the averaged fields <E>^{n+1}, <B>^{n+1} computed alongside are
what the next step gathers (they replace E, B in step 1).  The first step gathers
E^0, B^0.
"""
import numpy as np

from . import fdtd, grid, particles, psatd

STANDARD, GALILEAN, AVERAGED = 0, 1, 2
HYBRID, NODAL, STAGGERED, HYBRID_FDTD = 0, 1, 2, 3


class Params:
    """Grid and method parameters (the arguments of the problem statement, Sec. 4 and 5)."""

    def __init__(self, shape, dx, dt, shape_order, centering_order, variant=STANDARD,
                 v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0, filter_passes=0,
                 pusher=0, cycle=HYBRID):
        self.shape = tuple(int(n) for n in shape)
        self.dx = tuple(float(d) for d in dx)
        self.dt = float(dt)
        self.shape_order = int(shape_order)
        self.centering_order = tuple(int(o) for o in centering_order)
        self.variant = int(variant)
        self.v_gal = tuple(float(v) for v in v_gal) if variant != STANDARD else (0.0, 0.0, 0.0)
        self.spectral_order = tuple(int(o) for o in spectral_order)
        self.c = float(c)
        self.eps0 = float(eps0)
        self.filter_passes = int(filter_passes)
        self.pusher = int(pusher)        # 0: Boris, 1: Vay
        self.cycle = int(cycle)          # HYBRID (Sec. 2), the NODAL or STAGGERED comparison cycle,
                                         # or HYBRID_FDTD
        self._co = None
        self._k = None

    def fd_orders(self):
        """Finite-difference order per axis of the FDTD solver (0 -> 2, Yee)."""
        return tuple(o if o else 2 for o in self.spectral_order)

    def coefficients(self):
        if self._co is None:
            nodal = self.cycle == NODAL
            self._co = psatd.coefficients(self.shape, self.dx, self.dt, self.spectral_order,
                                          self.v_gal, self.c, self.eps0,
                                          averaged=self.variant == AVERAGED, nodal=nodal)
            self._k = psatd.staggered_k_grid(self.shape, self.dx, self.spectral_order, nodal=nodal)
        return self._co, self._k


def maxwell_update(p, E, B, J, rho_n, rho_np1):
    """Step 5: Yee E^n, B^n (real) -> Yee E^{n+1}, B^{n+1} and, if averaged, Yee <E>, <B>.

    Returns (E, B, avg or None, max |Im| seen in the inverse transforms).
    """
    co, k = p.coefficients()
    # positions of the components: the Yee grid, or the nodes in the nodal cycle
    nE = ("rho",) * 3 if p.cycle == NODAL else grid.E_NAMES
    nB = ("rho",) * 3 if p.cycle == NODAL else grid.B_NAMES
    nJ = ("rho",) * 3 if p.cycle == NODAL else grid.J_NAMES
    Eh = [grid.to_spectral(E[a], nE[a], p.dx) for a in range(3)]
    Bh = [grid.to_spectral(B[a], nB[a], p.dx) for a in range(3)]
    Jh = [grid.to_spectral(J[a], nJ[a], p.dx) for a in range(3)]
    rn = grid.to_spectral(rho_n, "rho", p.dx)
    rp = grid.to_spectral(rho_np1, "rho", p.dx)
    En, Bn = psatd.update(Eh, Bh, Jh, rn, rp, co, k, p.c)
    im = 0.0
    Eo, Bo = [], []
    for a in range(3):
        f, i1 = grid.from_spectral(En[a], nE[a], p.dx)
        g, i2 = grid.from_spectral(Bn[a], nB[a], p.dx)
        Eo.append(f)
        Bo.append(g)
        im = max(im, i1, i2)
    avg = None
    if p.variant == AVERAGED:
        Ea, Ba = psatd.update_averaged(Eh, Bh, Jh, rn, rp, co, k, p.c)
        avg = ([grid.from_spectral(Ea[a], nE[a], p.dx)[0] for a in range(3)],
               [grid.from_spectral(Ba[a], nB[a], p.dx)[0] for a in range(3)])
    return Eo, Bo, avg, im


def hybrid_step(p, state):
    """Advance `state` by one hybrid PIC step (in place on the dict, which is also returned).

    state: E (3 Yee arrays), B (3 Yee arrays), rho (nodal rho^n), species (list of
    dicts, see particles.push_and_deposit), optional 'avg' = (E_avg, B_avg) Yee
    arrays for the averaged variant.  Adds J (3 Yee arrays, J^{n+1/2}) and 'max_imag'.
    """
    gE, gB = state["E"], state["B"]
    if p.variant == AVERAGED and state.get("avg") is not None:
        gE, gB = state["avg"]
    o = p.centering_order
    if p.cycle in (NODAL, STAGGERED):   # comparison cycles: gather E, B where they live
        nE, nB = [np.asarray(f) for f in gE], [np.asarray(f) for f in gB]
    else:
        nE = [grid.center_to_nodal(gE[a], grid.E_NAMES[a], o) for a in range(3)]      # step 1
        nB = [grid.center_to_nodal(gB[a], grid.B_NAMES[a], o) for a in range(3)]
    Jn = [np.zeros(p.shape) for _ in range(3)]
    rho_np1 = np.zeros(p.shape)
    new_species = []
    for sp in state["species"]:                                                       # steps 2-3
        nsp, J, r = particles.push_and_deposit(sp, nE, nB, p.shape, p.dx, p.dt, p.shape_order,
                                               p.v_gal, p.c, p.pusher, staggered=p.cycle == STAGGERED)
        new_species.append(nsp)
        for a in range(3):
            Jn[a] += J[a]
        rho_np1 += r
    # optional smoothing of the deposits (Sec. 2): the solver sees the filtered rho^n, rho^{n+1}
    # and J; state["rho"] keeps the unfiltered deposit
    f = p.filter_passes
    Jf = [grid.bilinear_filter(Jn[a], f) for a in range(3)] if f else Jn
    rn_f = grid.bilinear_filter(state["rho"], f) if f else state["rho"]
    rp_f = grid.bilinear_filter(rho_np1, f) if f else rho_np1
    if p.cycle in (NODAL, STAGGERED):   # J already lives where the solver needs it
        Jy = Jf
    else:
        Jy = [grid.center_to_yee(Jf[a], grid.J_NAMES[a], o) for a in range(3)]         # step 4
    if p.cycle == HYBRID_FDTD:                                                        # step 5
        E, B = fdtd.yee_update(state["E"], state["B"], Jy, p.dt, p.fd_orders(), p.dx, p.c, p.eps0)
        avg, im = None, 0.0
    else:
        E, B, avg, im = maxwell_update(p, state["E"], state["B"], Jy, rn_f, rp_f)
    state.update(E=E, B=B, J=Jy, rho=rho_np1, species=new_species, max_imag=im)
    if avg is not None:
        state["avg"] = avg
    return state


def initial_rho(p, species):
    """rho^0 on the nodal grid from the initial particle positions."""
    rho = np.zeros(p.shape)
    for sp in species:
        rho += particles.deposit_rho(sp, p.shape, p.dx, p.shape_order)
    return rho
