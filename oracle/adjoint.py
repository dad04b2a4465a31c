"""Discrete adjoint (reverse mode) of the hybrid PSATD PIC step.

Test infrastructure only (see oracle/__init__.py).

The step (oracle.step.hybrid_step) is a composition of maps; the adjoint of the
step applies, in reverse order, the transpose (vector-Jacobian product) of each:

  1. centering E, B -> nodal (linear; Sec. 3): transpose = nodal -> staggered stencil
     (the two directions are transposes of each other, see grid.center_*);
  2. gather at x^n (linear in the nodal fields, B-spline in x): transpose = deposit of
     the force adjoints, plus the shape derivative for the position adjoint;
  3. Boris push (textbook rotation): reverse chain rule through its intermediates;
  4. v = u / gamma, x^{n+1/2} = x^n + dt (v - v_gal) / 2, x^{n+1} = x^n + dt (v - v_gal);
  5. deposit of J^{n+1/2} and rho^{n+1} (linear in q w v, B-spline in x): transpose =
     gather of the adjoint densities, plus the shape derivative;
  6. centering J nodal -> Yee (linear): transpose = staggered -> nodal stencil;
  7. PSATD update (linear in E, B, J, rho^n, rho^{n+1}; Sec. 4): per mode, the
     conjugate transpose of the update's coefficient matrix (the map is real, so
     its transpose is the per-mode conjugate transpose in the discrete Fourier basis).

The loss is the field energy of a probe box (Sec. 2 (iii)); the driver keeps a
checkpoint of the state every K steps and recomputes each segment forward before
running it backward.  Standard and Galilean variants; positions and momenta in FP64.
"""
import numpy as np

from . import grid, particles, psatd, step


# ---------------------------------------------------------------------------
# B-spline shapes and their derivatives (orders 1-3, as particles.shape_weights)
# ---------------------------------------------------------------------------

def shape_and_derivative(x, inv_dx, order):
    """(lowest node, weights[order+1, N], d weights / d x [order+1, N]) at positions x."""
    lo, w = particles.shape_weights(x, inv_dx, order)
    t = x * inv_dx
    base = np.floor(t + 0.5) if order == 2 else np.floor(t)
    d = t - base
    if order == 1:
        dw = np.stack([-np.ones_like(d), np.ones_like(d)])
    elif order == 2:
        dw = np.stack([-(0.5 - d), -2.0 * d, 0.5 + d])
    else:
        dw = np.stack([-0.5 * (1.0 - d) ** 2, (-12.0 * d + 9.0 * d * d) / 6.0,
                       (3.0 + 6.0 * d - 9.0 * d * d) / 6.0, 0.5 * d * d])
    return lo, w, dw * inv_dx


def _nodes(pos, shape, dx, order):
    """Per particle: index arrays, weight products and their gradient for every stencil node."""
    lo, w, dw = [], [], []
    for a in range(3):
        l, ww, dd = shape_and_derivative(pos[a], 1.0 / dx[a], order)
        lo.append(l)
        w.append(ww)
        dw.append(dd)
    for i in range(order + 1):
        for j in range(order + 1):
            for k in range(order + 1):
                idx = ((lo[0] + i) % shape[0], (lo[1] + j) % shape[1], (lo[2] + k) % shape[2])
                S = w[0][i] * w[1][j] * w[2][k]
                gS = (dw[0][i] * w[1][j] * w[2][k], w[0][i] * dw[1][j] * w[2][k], w[0][i] * w[1][j] * dw[2][k])
                yield idx, S, gS


def gather_with_gradient(fields, pos, dx, order):
    """F_c(x_p) and d F_c(x_p) / d x_a for nodal fields (list)."""
    shape = fields[0].shape
    val = [np.zeros_like(pos[0]) for _ in fields]
    grad = [[np.zeros_like(pos[0]) for _ in range(3)] for _ in fields]
    for idx, S, gS in _nodes(pos, shape, dx, order):
        for c, f in enumerate(fields):
            fv = f[idx]
            val[c] += S * fv
            for a in range(3):
                grad[c][a] += gS[a] * fv
    return val, grad


def deposit_values(shape, pos, values, dx, order):
    """sum_p values_p S(x_p - x_i) on nodal arrays (no 1/dV: the transpose of the gather)."""
    out = [np.zeros(shape) for _ in values]
    for idx, S, _ in _nodes(pos, shape, dx, order):
        for v, o in zip(values, out):
            np.add.at(o, idx, v * S)
    return out


# ---------------------------------------------------------------------------
# transposes of the linear grid maps
# ---------------------------------------------------------------------------

def center_to_nodal_T(nbar, name, orders):
    """Transpose of grid.center_to_nodal: the nodal -> staggered stencil along the same axes (z, y, x order)."""
    f = nbar
    for a in (2, 1, 0):
        if grid.STAG[name][a]:
            f = grid.center_nodal_to_staggered_1d(f, a, orders[a])
    return f


def center_to_yee_T(ybar, name, orders):
    """Transpose of grid.center_to_yee: the staggered -> nodal stencil."""
    f = ybar
    for a in (2, 1, 0):
        if grid.STAG[name][a]:
            f = grid.center_staggered_to_nodal_1d(f, a, orders[a])
    return f


def update_T(Ebar, Bbar, co, k, c=1.0):
    """Conjugate transpose of psatd.update, per mode, on paper-convention adjoint spectra.

    Forward (Sec. 4.3, theta = 1 in the standard case):
      B' = TC B - i TS K E + i X1 K J,
      E' = TC E + i c^2 TS K B + X4 J + i (TX3 rho^n - X2 rho^{n+1}) k,
    with K v = [k] x v (real, antisymmetric).  Returns (Ebar, Bbar, Jbar, rho_n_bar, rho_np1_bar).
    """
    cj = {key: np.conj(v) for key, v in co.items()}
    KB = psatd.cross(k, Bbar)
    KE = psatd.cross(k, Ebar)
    kdotE = k[0] * Ebar[0] + k[1] * Ebar[1] + k[2] * Ebar[2]
    Eo = [cj["TC"] * Ebar[a] - 1j * cj["TS"] * KB[a] for a in range(3)]
    Bo = [cj["TC"] * Bbar[a] + 1j * c * c * cj["TS"] * KE[a] for a in range(3)]
    Jo = [1j * cj["X1"] * KB[a] + cj["X4"] * Ebar[a] for a in range(3)]
    rn = -1j * cj["TX3"] * kdotE
    rp = 1j * cj["X2"] * kdotE
    return Eo, Bo, Jo, rn, rp


def maxwell_update_T(p, Ebar, Bbar):
    """Transpose of step.maxwell_update (the real-space field solve): adjoint Yee E', B'
    -> adjoints of E^n, B^n (Yee), J^{n+1/2} (Yee), rho^n, rho^{n+1} (nodal)."""
    co, k = p.coefficients()
    Eh = [grid.to_spectral(Ebar[a], grid.E_NAMES[a], p.dx) for a in range(3)]
    Bh = [grid.to_spectral(Bbar[a], grid.B_NAMES[a], p.dx) for a in range(3)]
    Eo, Bo, Jo, rn, rp = update_T(Eh, Bh, co, k, p.c)
    E = [grid.from_spectral(Eo[a], grid.E_NAMES[a], p.dx)[0] for a in range(3)]
    B = [grid.from_spectral(Bo[a], grid.B_NAMES[a], p.dx)[0] for a in range(3)]
    J = [grid.from_spectral(Jo[a], grid.J_NAMES[a], p.dx)[0] for a in range(3)]
    return E, B, J, grid.from_spectral(rn, "rho", p.dx)[0], grid.from_spectral(rp, "rho", p.dx)[0]


# ---------------------------------------------------------------------------
# Boris push and its reverse
# ---------------------------------------------------------------------------

def boris_T(u, E, B, q, m, dt, ubar_new, c=1.0):
    """Reverse of particles.boris: given the adjoint of u^{n+1/2}, return the adjoints of
    u^{n-1/2}, E_p and B_p (lists of 3 arrays)."""
    k = q * dt / (2.0 * m)
    um = [u[a] + k * E[a] for a in range(3)]
    gm = np.sqrt(1.0 + (um[0] ** 2 + um[1] ** 2 + um[2] ** 2) / (c * c))
    t = [k * B[a] / gm for a in range(3)]
    ts = 1.0 + t[0] ** 2 + t[1] ** 2 + t[2] ** 2
    s = [2.0 * t[a] / ts for a in range(3)]
    up = [um[0] + (um[1] * t[2] - um[2] * t[1]),
          um[1] + (um[2] * t[0] - um[0] * t[2]),
          um[2] + (um[0] * t[1] - um[1] * t[0])]
    cross = lambda a, b: [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    dot = lambda a, b: a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
    upl_bar = list(ubar_new)                        # u' = upl + k E
    Ebar = [k * ubar_new[a] for a in range(3)]
    um_bar = list(upl_bar)                          # upl = um + up x s
    sxa = cross(s, upl_bar)
    up_bar = sxa
    s_bar = cross(upl_bar, up)
    txa = cross(t, up_bar)                          # up = um + um x t
    um_bar = [um_bar[a] + up_bar[a] + txa[a] for a in range(3)]
    t_bar = cross(up_bar, um)
    sdt = dot(s_bar, t)                             # s = 2 t / (1 + t.t)
    t_bar = [t_bar[a] + 2.0 * s_bar[a] / ts - 4.0 * sdt / ts ** 2 * t[a] for a in range(3)]
    Bbar = [k / gm * t_bar[a] for a in range(3)]    # t = k B / gm
    gm_bar = -dot(t, t_bar) / gm
    um_bar = [um_bar[a] + gm_bar * um[a] / (c * c * gm) for a in range(3)]   # gm = sqrt(1 + um.um/c^2)
    ubar = list(um_bar)                             # um = u + k E
    Ebar = [Ebar[a] + k * um_bar[a] for a in range(3)]
    return ubar, Ebar, Bbar


# ---------------------------------------------------------------------------
# one adjoint step
# ---------------------------------------------------------------------------

def adjoint_step(p, state, adj):
    """Reverse of step.hybrid_step for the state at t^n.

    state: E, B (Yee), rho (rho^n), species (x^n, u^{n-1/2}) at step n.
    adj:   adjoints of the step's outputs: E, B (Yee), rho (rho^{n+1}), species_bar (per species
           dict with x, y, z, ux, uy, uz adjoints of x^{n+1}, u^{n+1/2}).
    Returns the adjoints of the inputs in the same layout (rho = adjoint of rho^n).
    Standard and Galilean variants (the averaged variant is not covered).
    """
    if p.variant == step.AVERAGED:
        raise NotImplementedError("adjoint of the averaged Galilean step is not provided")
    o = p.centering_order
    dV = p.dx[0] * p.dx[1] * p.dx[2]
    L = [p.shape[a] * p.dx[a] for a in range(3)]
    # 7: field update
    Eb, Bb, Jyb, rnb, rpb = maxwell_update_T(p, adj["E"], adj["B"])
    rpb = rpb + adj["rho"]                          # rho^{n+1} is also an output of the step
    # 6: centering J -> Yee
    Jnb = [center_to_yee_T(Jyb[a], grid.J_NAMES[a], o) for a in range(3)]
    # recompute the forward particle stage
    nE = [grid.center_to_nodal(state["E"][a], grid.E_NAMES[a], o) for a in range(3)]
    nB = [grid.center_to_nodal(state["B"][a], grid.B_NAMES[a], o) for a in range(3)]
    nEb = [np.zeros(p.shape) for _ in range(3)]
    nBb = [np.zeros(p.shape) for _ in range(3)]
    out_species = []
    for sp, spb in zip(state["species"], adj["species"]):
        pos = [sp["x"], sp["y"], sp["z"]]
        (Ep, Bp_) = (particles.gather(nE, pos, p.dx, p.shape_order), particles.gather(nB, pos, p.dx, p.shape_order))
        u = [sp["ux"], sp["uy"], sp["uz"]]
        un = particles.boris(u, Ep, Bp_, sp["q"], sp["m"], p.dt, p.c)
        g = np.sqrt(1.0 + (un[0] ** 2 + un[1] ** 2 + un[2] ** 2) / (p.c * p.c))
        v = [un[a] / g for a in range(3)]
        mid = [particles.wrap(pos[a] + 0.5 * p.dt * (v[a] - p.v_gal[a]), L[a]) for a in range(3)]
        new = [particles.wrap(pos[a] + p.dt * (v[a] - p.v_gal[a]), L[a]) for a in range(3)]
        qw = sp["q"] * sp["w"] / dV
        # 5: deposits
        Jm, Jgrad = gather_with_gradient(Jnb, mid, p.dx, p.shape_order)
        _, rgrad = gather_with_gradient([rpb], new, p.dx, p.shape_order)
        xnew_bar = [spb[k] + qw * rgrad[0][a] for a, k in enumerate(("x", "y", "z"))]
        xmid_bar = [qw * (v[0] * Jgrad[0][a] + v[1] * Jgrad[1][a] + v[2] * Jgrad[2][a]) for a in range(3)]
        v_bar = [qw * Jm[a] + 0.5 * p.dt * xmid_bar[a] + p.dt * xnew_bar[a] for a in range(3)]
        x_bar = [xnew_bar[a] + xmid_bar[a] for a in range(3)]
        # 4: v = u/gamma (symmetric Jacobian I/g - u u^T/(c^2 g^3))
        udotv = (un[0] * v_bar[0] + un[1] * v_bar[1] + un[2] * v_bar[2]) / (p.c * p.c * g ** 3)
        un_bar = [spb["u" + "xyz"[a]] + v_bar[a] / g - un[a] * udotv for a in range(3)]
        # 3: Boris
        u_bar, Ep_bar, Bp_bar = boris_T(u, Ep, Bp_, sp["q"], sp["m"], p.dt, un_bar, p.c)
        # 2: gather
        gE = deposit_values(p.shape, pos, Ep_bar, p.dx, p.shape_order)
        gB = deposit_values(p.shape, pos, Bp_bar, p.dx, p.shape_order)
        for a in range(3):
            nEb[a] += gE[a]
            nBb[a] += gB[a]
        _, Egrad = gather_with_gradient(nE, pos, p.dx, p.shape_order)
        _, Bgrad = gather_with_gradient(nB, pos, p.dx, p.shape_order)
        for a in range(3):
            x_bar[a] = x_bar[a] + sum(Ep_bar[c] * Egrad[c][a] + Bp_bar[c] * Bgrad[c][a] for c in range(3))
        out_species.append({"x": x_bar[0], "y": x_bar[1], "z": x_bar[2],
                            "ux": u_bar[0], "uy": u_bar[1], "uz": u_bar[2]})
    # 1: centering E, B -> nodal
    E_out = [Eb[a] + center_to_nodal_T(nEb[a], grid.E_NAMES[a], o) for a in range(3)]
    B_out = [Bb[a] + center_to_nodal_T(nBb[a], grid.B_NAMES[a], o) for a in range(3)]
    return {"E": E_out, "B": B_out, "rho": rnb, "species": out_species}


# ---------------------------------------------------------------------------
# loss and gradient with checkpointing
# ---------------------------------------------------------------------------

def probe_energy(p, E, B, lo, hi):
    """W over the probe box [lo, hi) of each Yee component (Sec. 2 (iii))."""
    mu0 = 1.0 / (p.eps0 * p.c * p.c)
    dV = p.dx[0] * p.dx[1] * p.dx[2]
    sl = tuple(slice(lo[a], hi[a]) for a in range(3))
    return 0.5 * dV * (p.eps0 * sum(float(np.sum(E[a][sl] ** 2)) for a in range(3))
                       + sum(float(np.sum(B[a][sl] ** 2)) for a in range(3)) / mu0)


def probe_energy_bar(p, E, B, lo, hi):
    mu0 = 1.0 / (p.eps0 * p.c * p.c)
    dV = p.dx[0] * p.dx[1] * p.dx[2]
    mask = np.zeros(p.shape)
    mask[tuple(slice(lo[a], hi[a]) for a in range(3))] = 1.0
    return [p.eps0 * dV * E[a] * mask for a in range(3)], [dV / mu0 * B[a] * mask for a in range(3)]


def _copy_state(st):
    return {"E": [a.copy() for a in st["E"]], "B": [a.copy() for a in st["B"]], "rho": st["rho"].copy(),
            "species": [{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
                        for s in st["species"]]}


def loss_and_gradient(p, state0, nsteps, lo, hi, checkpoint=10):
    """Probe-box field energy after nsteps and its gradient w.r.t. the initial state.

    Returns (loss, adjoint dict at step 0: E, B, rho, species with x..uz adjoints).
    """
    ckpt = {}
    st = _copy_state(state0)
    for n in range(nsteps):
        if n % checkpoint == 0:
            ckpt[n] = _copy_state(st)
        step.hybrid_step(p, st)
    loss = probe_energy(p, st["E"], st["B"], lo, hi)
    Eb, Bb = probe_energy_bar(p, st["E"], st["B"], lo, hi)
    adj = {"E": Eb, "B": Bb, "rho": np.zeros(p.shape),
           "species": [{k: np.zeros_like(s["x"]) for k in ("x", "y", "z", "ux", "uy", "uz")}
                       for s in state0["species"]]}
    starts = sorted(ckpt)
    for s0 in reversed(starts):
        s1 = min(s0 + checkpoint, nsteps)
        states = [_copy_state(ckpt[s0])]
        for n in range(s0, s1 - 1):
            nxt = _copy_state(states[-1])
            step.hybrid_step(p, nxt)
            states.append(nxt)
        for n in range(s1 - 1, s0 - 1, -1):
            adj = adjoint_step(p, states[n - s0], adj)
    return loss, adj
