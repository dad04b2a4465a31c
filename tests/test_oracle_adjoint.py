"""Pins for oracle.adjoint: every transpose is checked by a dot-product test against the
forward map it reverses, Boris by finite differences, and the full reverse pass by
central finite differences of the oracle's own forward step (directional derivatives
with respect to the initial momenta and to the amplitude of the initial E field)."""
import numpy as np
import pytest

from oracle import adjoint, grid, particles, step
from paper_2106_12919_gb300 import workloads


def _params(shape=(8, 8, 16), order=1, variant=0, v=(0.0, 0.0, 0.0), sorder=(0, 0, 0)):
    return step.Params(shape, (1.0, 0.8, 0.5), 0.4, order, (4, 4, 8), variant, v, sorder)


@pytest.mark.parametrize("variant,v,sorder", [(0, (0, 0, 0), (0, 0, 0)), (1, (0, 0, 0.8), (8, 8, 8))])
def test_maxwell_transpose_dot_product(variant, v, sorder):
    p = _params(variant=variant, v=v, sorder=sorder)
    rng = np.random.default_rng(0)
    r = lambda: rng.normal(size=p.shape)
    E, B, J = [r() for _ in range(3)], [r() for _ in range(3)], [r() for _ in range(3)]
    rn, rp = r(), r()
    Eb, Bb = [r() for _ in range(3)], [r() for _ in range(3)]
    Eo, Bo, _, _ = step.maxwell_update(p, E, B, J, rn, rp)
    lhs = sum(np.sum(Eb[a] * Eo[a]) + np.sum(Bb[a] * Bo[a]) for a in range(3))
    tE, tB, tJ, trn, trp = adjoint.maxwell_update_T(p, Eb, Bb)
    rhs = sum(np.sum(tE[a] * E[a]) + np.sum(tB[a] * B[a]) + np.sum(tJ[a] * J[a]) for a in range(3)) \
        + np.sum(trn * rn) + np.sum(trp * rp)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_centering_transposes_dot_product():
    rng = np.random.default_rng(1)
    shape, orders = (8, 8, 16), (4, 6, 8)
    for name in grid.E_NAMES + grid.B_NAMES:
        x, y = rng.normal(size=shape), rng.normal(size=shape)
        lhs = np.sum(y * grid.center_to_nodal(x, name, orders))
        rhs = np.sum(adjoint.center_to_nodal_T(y, name, orders) * x)
        assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(x) * 10)
    for name in grid.J_NAMES:
        x, y = rng.normal(size=shape), rng.normal(size=shape)
        lhs = np.sum(y * grid.center_to_yee(x, name, orders))
        rhs = np.sum(adjoint.center_to_yee_T(y, name, orders) * x)
        assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(x) * 10)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_shape_derivative_matches_finite_difference(order):
    rng = np.random.default_rng(order)
    x = rng.uniform(1, 10, 500)
    lo, w, dw = adjoint.shape_and_derivative(x, 2.0, order)
    h = 1e-7
    lo2, w2, _ = adjoint.shape_and_derivative(x + h, 2.0, order)
    lo1, w1, _ = adjoint.shape_and_derivative(x - h, 2.0, order)
    ok = (lo1 == lo) & (lo2 == lo)
    np.testing.assert_allclose(((w2 - w1) / (2 * h))[:, ok], dw[:, ok], atol=1e-6)


def test_boris_reverse_matches_finite_difference():
    rng = np.random.default_rng(3)
    n = 50
    u = [rng.normal(0, 0.5, n) for _ in range(3)]
    E = [rng.normal(0, 1.0, n) for _ in range(3)]
    B = [rng.normal(0, 2.0, n) for _ in range(3)]
    ub = [rng.normal(size=n) for _ in range(3)]
    q, m, dt = -1.0, 1.3, 0.3
    gu, gE, gB = adjoint.boris_T(u, E, B, q, m, dt, ub)
    f = lambda uu, EE, BB: sum(ub[a] * particles.boris(uu, EE, BB, q, m, dt)[a] for a in range(3))
    h = 1e-6
    for which, grad in ((0, gu), (1, gE), (2, gB)):
        for a in range(3):
            args_p = [list(u), list(E), list(B)]
            args_m = [list(u), list(E), list(B)]
            args_p[which][a] = args_p[which][a] + h
            args_m[which][a] = args_m[which][a] - h
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            np.testing.assert_allclose(grad[a], fd, rtol=1e-6, atol=1e-8)


def _seed_state(order, shape=(8, 8, 16), ppc=2, steps=None):
    w = workloads.seed_wave(shape=shape, ppc=ppc, amplitude=0.05, u_th=0.05)
    prm = dict(w["params"])
    prm["shape_order"] = order
    p = step.Params(**prm)
    st = {"E": w["E"], "B": w["B"], "species": w["species"]}
    st["rho"] = step.initial_rho(p, st["species"])
    profile = w["E"][0] / 0.05
    return p, st, profile


@pytest.mark.parametrize("order", [1, 3])
def test_full_reverse_pass_matches_central_differences(order):
    p, st0, profile = _seed_state(order)
    lo, hi = (2, 2, 4), (6, 6, 12)
    nsteps = 4
    loss, adj = adjoint.loss_and_gradient(p, st0, nsteps, lo, hi, checkpoint=3)

    def L(du=None, dA=0.0):
        st = adjoint._copy_state(st0)
        st["E"][0] = st["E"][0] + dA * profile
        if du is not None:
            for k in ("ux", "uy", "uz"):
                st["species"][0][k] = st["species"][0][k] + du[k]
        for _ in range(nsteps):
            step.hybrid_step(p, st)
        return adjoint.probe_energy(p, st["E"], st["B"], lo, hi)

    assert abs(L() - loss) < 1e-14 * loss
    rng = np.random.default_rng(11)
    n = st0["species"][0]["x"].size
    d = {k: rng.normal(size=n) for k in ("ux", "uy", "uz")}
    eps = 1e-6
    fd = (L({k: eps * v for k, v in d.items()}) - L({k: -eps * v for k, v in d.items()})) / (2 * eps)
    ad = sum(np.sum(adj["species"][0][k] * d[k]) for k in ("ux", "uy", "uz"))
    assert abs(fd - ad) < 1e-6 * abs(ad)
    fdA = (L(dA=eps) - L(dA=-eps)) / (2 * eps)
    adA = np.sum(adj["E"][0] * profile)
    assert abs(fdA - adA) < 1e-6 * abs(adA)
