"""The oracle's pins reject wrong oracles: each case swaps one oracle function for a plausible
mistake (on the CPU, for the duration of the case) and checks that the pin written for that
function fails.  A pin that passed a wrong oracle would not pin anything."""
import numpy as np
import pytest

import test_oracle_fdtd as T_fdtd
import test_oracle_grid as T_grid
import test_oracle_particles as T_particles
import test_oracle_psatd as T_psatd
from oracle import fdtd, grid, particles, psatd


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_boris_with_the_rotation_reversed(monkeypatch):
    orig = particles.boris
    monkeypatch.setattr(particles, "boris", lambda u, E, B, q, m, dt, c=1.0: orig(u, E, [-b for b in B], q, m, dt, c))
    _fails(T_particles.test_boris_pure_magnetic_gyration)


def test_cubic_shape_with_two_weights_swapped(monkeypatch):
    orig = particles.shape_weights

    def wrong(x, inv_dx, order, offset=0.0):
        lo, w = orig(x, inv_dx, order, offset)
        return lo, (w[[0, 2, 1, 3]] if order == 3 else w)
    monkeypatch.setattr(particles, "shape_weights", wrong)
    _fails(T_particles.test_shape_weights_are_bsplines, 3)


def test_galilean_move_with_the_wrong_sign(monkeypatch):
    orig = particles.push_and_deposit

    def wrong(sp, E, B, shape, dx, dt, order, v_gal=(0.0, 0.0, 0.0), *a, **k):
        return orig(sp, E, B, shape, dx, dt, order, tuple(-v for v in v_gal), *a, **k)
    monkeypatch.setattr(particles, "push_and_deposit", wrong)
    _fails(T_particles.test_galilean_drift_and_midpoint_current, 1)


def test_centering_shifted_by_one_node(monkeypatch):
    orig = grid.center_staggered_to_nodal_1d
    monkeypatch.setattr(grid, "center_staggered_to_nodal_1d",
                        lambda f, axis, order: np.roll(orig(f, axis, order), 1, axis=axis))
    _fails(T_grid.test_centering_on_single_mode_is_zeta, 4)


def test_psatd_update_with_rho_n_and_rho_np1_swapped(monkeypatch):
    orig = psatd.update
    monkeypatch.setattr(psatd, "update", lambda Eh, Bh, Jh, rn, rp, co, k, c=1.0: orig(Eh, Bh, Jh, rp, rn, co, k, c))
    _fails(T_psatd.test_update_matches_exact_ode_solution, T_psatd.CASES[0])


def test_psatd_update_with_the_current_dropped(monkeypatch):
    orig = psatd.update
    monkeypatch.setattr(psatd, "update",
                        lambda Eh, Bh, Jh, rn, rp, co, k, c=1.0: orig(Eh, Bh, [0 * j for j in Jh], rn, rp, co, k, c))
    _fails(T_psatd.test_update_matches_exact_ode_solution, T_psatd.CASES[0])


def test_fdtd_difference_at_the_wrong_half_point(monkeypatch):
    orig = fdtd.d_to_half
    monkeypatch.setattr(fdtd, "d_to_half", lambda f, axis, order, dx: np.roll(orig(f, axis, order, dx), 1, axis=axis))
    _fails(T_fdtd.test_derivative_of_a_mode, 2, 0)


def test_fdtd_without_the_current(monkeypatch):
    orig = fdtd.yee_update
    monkeypatch.setattr(fdtd, "yee_update", lambda E, B, J, *a, **k: orig(E, B, [0 * j for j in J], *a, **k))
    _fails(T_fdtd.test_div_curl_zero_and_gauss, (2, 2, 2))
