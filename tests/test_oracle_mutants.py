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


def test_current_deposited_at_the_new_position(monkeypatch):
    # J^{n+1/2} belongs at the midpoint x^n + dt (v - v_gal) / 2 (Sec. 2), not at x^{n+1}
    orig = particles.push_and_deposit

    def wrong(sp, E, B, shape, dx, dt, order, v_gal=(0.0, 0.0, 0.0), c=1.0, *a, **k):
        out, _, rho = orig(sp, E, B, shape, dx, dt, order, v_gal, c, *a, **k)
        g = np.sqrt(1.0 + (out["ux"] ** 2 + out["uy"] ** 2 + out["uz"] ** 2) / (c * c))
        qw = sp["q"] * sp["w"]
        J = particles.deposit(shape, [out["x"], out["y"], out["z"]],
                              [qw * out["ux"] / g, qw * out["uy"] / g, qw * out["uz"] / g], dx, order)
        return out, J, rho
    monkeypatch.setattr(particles, "push_and_deposit", wrong)
    _fails(T_particles.test_galilean_drift_and_midpoint_current, 2)


def test_charge_deposited_at_the_midpoint(monkeypatch):
    # rho^{n+1} belongs at x^{n+1}
    orig = particles.push_and_deposit

    def wrong(sp, E, B, shape, dx, dt, order, v_gal=(0.0, 0.0, 0.0), c=1.0, *a, **k):
        out, J, _ = orig(sp, E, B, shape, dx, dt, order, v_gal, c, *a, **k)
        mid = [0.5 * (sp[key] + out[key]) for key in ("x", "y", "z")]
        (rho,) = particles.deposit(shape, mid, [sp["q"] * sp["w"]], dx, order)
        return out, J, rho
    monkeypatch.setattr(particles, "push_and_deposit", wrong)
    _fails(T_particles.test_galilean_drift_and_midpoint_current, 3)


def test_deposit_without_the_cell_volume(monkeypatch):
    orig = particles.deposit
    monkeypatch.setattr(particles, "deposit",
                        lambda gs, pos, vals, dx, order, offset=(0.0, 0.0, 0.0):
                        [d * np.prod(dx) for d in orig(gs, pos, vals, dx, order, offset)])
    _fails(T_particles.test_deposit_gather_adjoint_and_charge, 3)


def test_boris_rotation_without_gamma(monkeypatch):
    # the non-relativistic rotation angle q B dt / m in place of q B dt / (m gamma)
    orig = particles.boris
    monkeypatch.setattr(particles, "boris", lambda u, E, B, q, m, dt, c=1.0: orig(u, E, B, q, m, dt, 1e150))
    _fails(T_particles.test_boris_pure_magnetic_gyration)


def test_vay_with_the_rotation_reversed(monkeypatch):
    orig = particles.vay
    monkeypatch.setattr(particles, "vay", lambda u, E, B, q, m, dt, c=1.0: orig(u, E, [-b for b in B], q, m, dt, c))
    _fails(T_particles.test_vay_solves_its_defining_equation)


def test_staggered_fornberg_coefficients_without_the_alternating_sign(monkeypatch):
    import test_oracle_fornberg as T_fornberg
    from oracle import fornberg
    orig = fornberg.alpha_staggered
    monkeypatch.setattr(fornberg, "alpha_staggered", lambda m: [abs(a) for a in orig(m)])
    _fails(T_fornberg.test_staggered_moment_property, 2)


def test_centered_wave_number_in_place_of_the_staggered_one(monkeypatch):
    import test_oracle_fornberg as T_fornberg
    from oracle import fornberg
    monkeypatch.setattr(fornberg, "k_staggered", fornberg.k_centered)
    _fails(T_fornberg.test_modified_wave_numbers_order2_closed_form)


def test_centering_symbol_applied_twice(monkeypatch):
    import test_oracle_fornberg as T_fornberg
    from oracle import fornberg
    orig = fornberg.zeta
    monkeypatch.setattr(fornberg, "zeta", lambda N, order: orig(N, order) ** 2)
    _fails(T_fornberg.test_zeta_special_values_and_limit)


def test_half_cell_phase_with_the_wrong_sign(monkeypatch):
    orig = grid.shift_factor
    monkeypatch.setattr(grid, "shift_factor", lambda shape, dx, stag, sign: orig(shape, dx, stag, -sign))
    _fails(T_grid.test_spectral_convention_matches_direct_sum, "Ex")


def test_averaged_update_without_the_time_average(monkeypatch):
    monkeypatch.setattr(psatd, "update_averaged", psatd.update)
    _fails(T_psatd.test_update_matches_exact_ode_solution, T_psatd.CASES[3])


def test_galilean_coefficients_with_the_velocity_reversed(monkeypatch):
    orig = psatd.coefficients

    def wrong(shape, dx, dt, spectral_order, v_gal=(0.0, 0.0, 0.0), *a, **k):
        return orig(shape, dx, dt, spectral_order, tuple(-v for v in v_gal), *a, **k)
    monkeypatch.setattr(psatd, "coefficients", wrong)
    _fails(T_psatd.test_update_matches_exact_ode_solution, T_psatd.CASES[5])


def test_filter_with_one_pass_too_many(monkeypatch):
    orig = grid.bilinear_filter
    monkeypatch.setattr(grid, "bilinear_filter", lambda f, passes: orig(f, passes + 1))
    _fails(T_grid.test_bilinear_filter_symbol_sum_and_stencil)


def test_field_energy_without_the_half(monkeypatch):
    import test_oracle_diagnostics as T_diag
    from oracle import diagnostics
    orig = diagnostics.field_energy
    monkeypatch.setattr(diagnostics, "field_energy", lambda *a, **k: 2.0 * orig(*a, **k))
    _fails(T_diag.test_field_energy_uniform_fields_closed_form)


def test_boris_reverse_with_the_rotation_reversed(monkeypatch):
    import test_oracle_adjoint as T_adj
    from oracle import adjoint
    orig = adjoint.boris_T
    monkeypatch.setattr(adjoint, "boris_T",
                        lambda u, E, B, q, m, dt, ub, c=1.0: orig(u, E, [-b for b in B], q, m, dt, ub, c))
    _fails(T_adj.test_boris_reverse_matches_finite_difference)


def test_update_transpose_without_the_conjugate(monkeypatch):
    # a plain transpose of the Galilean update (complex coefficients) is not its adjoint
    import test_oracle_adjoint as T_adj
    from oracle import adjoint
    orig = adjoint.update_T
    monkeypatch.setattr(adjoint, "update_T", lambda Eb, Bb, co, k, c=1.0:
                        orig(Eb, Bb, {key: np.conj(v) for key, v in co.items()}, k, c))
    _fails(T_adj.test_maxwell_transpose_dot_product, 1, (0, 0, 0.8), (8, 8, 8))


def test_fields_gathered_without_centering(monkeypatch):
    # Yee E, B read as if they were nodal: a half-cell staggering error the mirror symmetry exposes
    import test_oracle_symmetry as T_sym
    monkeypatch.setattr(grid, "center_to_nodal", lambda f, name, orders: np.asarray(f))
    _fails(T_sym.test_mirror_reflection_x, 0, 0.0, 2, 0)


def test_current_solved_without_centering(monkeypatch):
    import test_oracle_symmetry as T_sym
    monkeypatch.setattr(grid, "center_to_yee", lambda f, name, orders: np.asarray(f))
    _fails(T_sym.test_mirror_reflection_x, 0, 0.0, 2, 0)


def test_curl_with_one_component_sign_flipped(monkeypatch):
    import test_oracle_step as T_step
    orig = psatd.cross

    def wrong(k, F):
        r = orig(k, F)
        return [r[0], -r[1], r[2]]
    monkeypatch.setattr(psatd, "cross", wrong)
    _fails(T_step.test_vacuum_energy_conserved, 0, (0, 0, 0), 0.0)
