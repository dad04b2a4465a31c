"""Exact symmetries of the whole hybrid cycle (oracle.step): the method commutes with the mirror
reflection x -> -x, with the exchange of the x and y axes, and with a translation by one cell.

Under a reflection E and J are polar vectors and B an axial one; on the grid a component
staggered along the reflected axis maps index i -> N-1-i, a nodal one i -> -i (mod N).  The
exchange of two axes is an improper rotation as well (B picks up a sign).  These are symmetries of
the continuous equations and of every discrete operator of the cycle (symmetric Fornberg
centering, B-spline shapes, the k-space update on a symmetric k grid, the FDTD differences, the
Boris push), so running
the cycle on the transformed state must give the transformed result, to rounding.  A staggering
offset, a phase sign, an axis mix-up or a one-sided stencil anywhere in the cycle breaks them."""
import numpy as np
import pytest

from oracle import grid, step
from paper_2106_12919_gb300 import workloads

def _reflect(a, name, ax=0):
    """Mirror along axis `ax` of the array of component `name` (E/B/J + x/y/z, or rho)."""
    stag = grid.STAG[name][ax]
    f = np.flip(a, axis=ax)
    f = f if stag else np.roll(f, 1, axis=ax)
    kind, comp = (name[0], name[1:]) if name != "rho" else ("rho", "")
    along = comp == "xyz"[ax]
    if kind in ("E", "J"):        # polar: the component along the mirror axis flips
        sgn = -1.0 if along else 1.0
    elif kind == "B":             # axial: the two other components flip
        sgn = 1.0 if along else -1.0
    else:
        sgn = 1.0
    return sgn * f


def _reflect_x(a, name):
    return _reflect(a, name, 0)


def _state(seed, shape=(8, 8, 16), ppc=2, variant=0, v=0.0, order=2, cycle=step.HYBRID):
    w = workloads.thermal_plasma(shape=shape, ppc=ppc, u_th=0.05)
    p = dict(w["params"])
    p.update(dx=(0.5, 0.5, 0.25), dt=0.2, shape_order=order, centering_order=(4, 4, 8), variant=variant,
             v_gal=(0.0, 0.0, v), spectral_order=(8, 8, 16) if variant else (0, 0, 0))
    rng = np.random.default_rng(seed)
    E = [0.05 * rng.normal(size=shape) for _ in range(3)]
    B = [0.05 * rng.normal(size=shape) for _ in range(3)]
    sp = [dict(s) for s in w["species"]]
    return step.Params(**p, cycle=cycle), E, B, sp


def _run(prm, E, B, sp, nsteps=2):
    st = {"E": [a.copy() for a in E], "B": [a.copy() for a in B], "species": [dict(s) for s in sp]}
    st["rho"] = step.initial_rho(prm, st["species"])
    for _ in range(nsteps):
        step.hybrid_step(prm, st)
    return st


def _close(a, b, scale):
    assert np.max(np.abs(a - b)) < 1e-12 * scale


@pytest.mark.parametrize("variant,v,order,cycle", [(0, 0.0, 1, 0), (0, 0.0, 2, 0), (0, 0.0, 3, 0), (1, 0.6, 2, 0),
                                                   (2, 0.5, 3, 0), (0, 0.0, 2, step.STAGGERED),
                                                   (0, 0.0, 3, step.HYBRID_FDTD)])
def test_mirror_reflection_x(variant, v, order, cycle):
    prm, E, B, sp = _state(1, variant=variant, v=v, order=order, cycle=cycle)
    L = prm.shape[0] * prm.dx[0]
    ref = _run(prm, E, B, sp)
    Er = [_reflect_x(E[a], grid.E_NAMES[a]) for a in range(3)]
    Br = [_reflect_x(B[a], grid.B_NAMES[a]) for a in range(3)]
    spr = []
    for s in sp:
        t = dict(s)
        t["x"] = np.mod(L - s["x"], L)
        t["ux"] = -s["ux"]
        spr.append(t)
    got = _run(prm, Er, Br, spr)
    sE = max(np.abs(e).max() for e in ref["E"])
    sB = max(np.abs(b).max() for b in ref["B"])
    sJ = max(np.abs(j).max() for j in ref["J"])
    for a in range(3):
        _close(got["E"][a], _reflect_x(ref["E"][a], grid.E_NAMES[a]), sE)
        _close(got["B"][a], _reflect_x(ref["B"][a], grid.B_NAMES[a]), sB)
        _close(got["J"][a], _reflect_x(ref["J"][a], grid.J_NAMES[a]), sJ)
    _close(got["rho"], _reflect_x(ref["rho"], "rho"), np.abs(ref["rho"]).max())
    for g, r in zip(got["species"], ref["species"]):
        dxp = np.mod(g["x"] - (L - r["x"]) + 0.5 * L, L) - 0.5 * L
        assert np.max(np.abs(dxp)) < 1e-12 * L
        _close(g["ux"], -r["ux"], 1.0)
        _close(g["uy"], r["uy"], 1.0)


@pytest.mark.parametrize("ax", [1, 2])
def test_mirror_reflection_y_and_z(ax):
    prm, E, B, sp = _state(4 + ax, order=3)
    L = prm.shape[ax] * prm.dx[ax]
    ref = _run(prm, E, B, sp)
    Er = [_reflect(E[a], grid.E_NAMES[a], ax) for a in range(3)]
    Br = [_reflect(B[a], grid.B_NAMES[a], ax) for a in range(3)]
    k, uk = "xyz"[ax], "u" + "xyz"[ax]
    spr = []
    for s in sp:
        t = dict(s)
        t[k] = np.mod(L - s[k], L)
        t[uk] = -s[uk]
        spr.append(t)
    got = _run(prm, Er, Br, spr)
    sE = max(np.abs(e).max() for e in ref["E"])
    sB = max(np.abs(b).max() for b in ref["B"])
    for a in range(3):
        _close(got["E"][a], _reflect(ref["E"][a], grid.E_NAMES[a], ax), sE)
        _close(got["B"][a], _reflect(ref["B"][a], grid.B_NAMES[a], ax), sB)
    _close(got["rho"], _reflect(ref["rho"], "rho", ax), np.abs(ref["rho"]).max())


def test_exchange_of_x_and_y():
    prm, E, B, sp = _state(2, order=3)
    ref = _run(prm, E, B, sp)
    sw = lambda a: np.swapaxes(a, 0, 1).copy()
    Es = [sw(E[1]), sw(E[0]), sw(E[2])]
    Bs = [-sw(B[1]), -sw(B[0]), -sw(B[2])]          # axial vector: the exchange is improper
    sps = []
    for s in sp:
        t = dict(s)
        t["x"], t["y"], t["ux"], t["uy"] = s["y"], s["x"], s["uy"], s["ux"]
        sps.append(t)
    got = _run(prm, Es, Bs, sps)
    sE = max(np.abs(e).max() for e in ref["E"])
    sB = max(np.abs(b).max() for b in ref["B"])
    _close(got["E"][0], sw(ref["E"][1]), sE)
    _close(got["E"][1], sw(ref["E"][0]), sE)
    _close(got["E"][2], sw(ref["E"][2]), sE)
    _close(got["B"][0], -sw(ref["B"][1]), sB)
    _close(got["B"][1], -sw(ref["B"][0]), sB)
    _close(got["B"][2], -sw(ref["B"][2]), sB)
    _close(got["rho"], sw(ref["rho"]), np.abs(ref["rho"]).max())


def test_translation_by_one_cell():
    prm, E, B, sp = _state(3, order=2)
    L = prm.shape[2] * prm.dx[2]
    ref = _run(prm, E, B, sp)
    sh = lambda a: np.roll(a, 1, axis=2)
    spt = []
    for s in sp:
        t = dict(s)
        t["z"] = np.mod(s["z"] + prm.dx[2], L)
        spt.append(t)
    got = _run(prm, [sh(e) for e in E], [sh(b) for b in B], spt)
    sE = max(np.abs(e).max() for e in ref["E"])
    for a in range(3):
        _close(got["E"][a], sh(ref["E"][a]), sE)
    _close(got["rho"], sh(ref["rho"]), np.abs(ref["rho"]).max())
