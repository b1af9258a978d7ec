"""Planted mistakes in the oracle, on the CPU (monkeypatch, undone after each
test): every slip below is a plausible error in restating the paper (a swapped
digit of a printed constant, a wrong coefficient, a dropped factor, a wrong sign,
transposed weights, the wrong Schwarz combination), and each makes one of the
oracle's pins fail. So the pins check the oracle against the paper and the
mathematics, not against its own formulas."""
import numpy as np
import pytest

from oracle import discretization as disc
from oracle import eos
from oracle import multilevel as ml
from oracle import newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn

import test_oracle_discretization as T_disc
import test_oracle_eos as T_eos
import test_oracle_krylov_newton as T_kn
import test_oracle_multilevel as T_ml
import test_oracle_schwarz as T_sch


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_swapped_digit_in_omega_a(monkeypatch):
    orig = eos.pr_constants
    monkeypatch.setattr(eos, "pr_constants", lambda f: (orig(f)[0] * 0.45742 / 0.45724, orig(f)[1]))
    _fails(T_eos.test_pr_constants_at_the_critical_point, syn.Fluid())


def test_swapped_digit_in_omega_b(monkeypatch):
    orig = eos.pr_constants
    monkeypatch.setattr(eos, "pr_constants", lambda f: (orig(f)[0], orig(f)[1] * 0.0787 / 0.0778))
    _fails(T_eos.test_pr_constants_at_the_critical_point, syn.Fluid())


def test_wrong_m_coefficient(monkeypatch):
    orig = eos.m_of_omega
    monkeypatch.setattr(eos, "m_of_omega", lambda w: orig(w) + 0.01)
    _fails(T_eos.test_m_of_omega_reproduces_the_acentric_factor, 0.2)


def test_bdf2_without_its_half(monkeypatch):
    orig = disc.bdf_terms

    def bad(p, p_l, p_lm1, dt, order):
        if order == 1:
            return orig(p, p_l, p_lm1, dt, order)
        return (3.0 * p - 4.0 * p_l + p_lm1) / dt, 3.0 / dt
    monkeypatch.setattr(disc, "bdf_terms", bad)
    _fails(T_disc.test_bdf_terms_exact_on_polynomials_in_time)


def test_bdf2_wrong_sign_on_the_older_level(monkeypatch):
    orig = disc.bdf_terms

    def bad(p, p_l, p_lm1, dt, order):
        if order == 1:
            return orig(p, p_l, p_lm1, dt, order)
        return (3.0 * p - 4.0 * p_l - p_lm1) / (2.0 * dt), 1.5 / dt
    monkeypatch.setattr(disc, "bdf_terms", bad)
    _fails(T_disc.test_bdf_terms_exact_on_polynomials_in_time)


def test_transmissibility_without_half_cells(monkeypatch):
    orig = disc.face_transmissibilities
    monkeypatch.setattr(disc, "face_transmissibilities",
                        lambda g, kx, ky, kz: tuple(2.0 * t for t in orig(g, kx, ky, kz)))
    _fails(T_disc.test_transmissibility_uniform_equals_kA_over_h)


def test_arithmetic_instead_of_harmonic_face_permeability(monkeypatch):
    def bad(grid, kx, ky, kz):
        nx, ny, nz = grid.nx, grid.ny, grid.nz
        K = [np.asarray(k, dtype=np.float64).reshape(nz, ny, nx) for k in (kx, ky, kz)]
        T = [np.zeros((nz, ny, nx)) for _ in range(3)]
        T[0][:, :, :-1] = grid.hy * grid.hz * 0.5 * (K[0][:, :, :-1] + K[0][:, :, 1:]) / grid.hx
        T[1][:, :-1, :] = grid.hx * grid.hz * 0.5 * (K[1][:, :-1, :] + K[1][:, 1:, :]) / grid.hy
        T[2][:-1, :, :] = grid.hx * grid.hy * 0.5 * (K[2][:-1, :, :] + K[2][1:, :, :]) / grid.hz
        return tuple(t.reshape(-1) for t in T)
    monkeypatch.setattr(disc, "face_transmissibilities", bad)
    _fails(T_disc.test_ideal_gas_steady_heterogeneous_series_resistance)


def test_interpolation_weights_swapped(monkeypatch):
    orig = ml.interp_1d

    def bad(n, r, order):
        P = np.array(orig(n, r, order), dtype=np.float64)
        for i in range(P.shape[0]):
            nz = np.nonzero(P[i])[0]
            if len(nz) == 2:
                P[i, nz] = P[i, nz[::-1]]
        return P
    monkeypatch.setattr(ml, "interp_1d", bad)
    _fails(T_ml.test_ratio_two_linear_weights)
    _fails(T_ml.test_polynomial_reproduction, 32, 4)


def test_line_search_step_off(monkeypatch):
    orig = newton.backtrack_lambda
    monkeypatch.setattr(newton, "backtrack_lambda", lambda *a: 0.9 * orig(*a))
    _fails(T_kn.test_backtrack_quadratic_step_is_exact_minimiser)
    _fails(T_kn.test_backtrack_cubic_step_is_exact_minimiser)


def test_left_ras_combined_as_classical_as(monkeypatch):
    orig = schwarz.Schwarz.apply

    def bad(self, r):
        if self.kind != schwarz.LEFT_RAS:
            return orig(self, r)
        self.kind = schwarz.AS
        try:
            return orig(self, r)
        finally:
            self.kind = schwarz.LEFT_RAS
    monkeypatch.setattr(schwarz.Schwarz, "apply", bad)
    _fails(T_sch.test_left_ras_transpose_is_right_ras_of_transpose)


def test_keys_kernel_with_another_parameter(monkeypatch):
    def bad(s):                  # cubic convolution with a = -3/4 instead of -1/2
        s = abs(s)
        if s < 1.0:
            return 1.25 * s ** 3 - 2.25 * s ** 2 + 1.0
        if s < 2.0:
            return -0.75 * s ** 3 + 3.75 * s ** 2 - 6.0 * s + 3.0
        return 0.0
    monkeypatch.setattr(ml, "keys_w", bad)
    _fails(T_ml.test_polynomial_reproduction, 32, 4)


def test_dz_dp_with_the_wrong_sign(monkeypatch):
    orig = eos.dz_dp_paper
    monkeypatch.setattr(eos, "dz_dp_paper", lambda *a: -orig(*a))
    _fails(T_eos.test_dz_dp_closed_form, syn.Fluid())


def test_gravity_term_with_the_wrong_sign(monkeypatch):
    import test_oracle_gravity as T_grav
    orig = disc.Problem.__init__

    def bad(self, res):
        orig(self, res)
        self.gravity = -self.gravity
    monkeypatch.setattr(disc.Problem, "__init__", bad)
    _fails(T_grav.test_closed_column_settles_to_the_hydrostatic_profile)


def test_vcycle_without_post_smoothing(monkeypatch):
    orig = ml.TwoLevel.apply

    def bad(self, r):
        if self.kind != ml.VCYCLE:
            return orig(self, r)
        e1 = self.M(r)
        return e1 + self.coarse(r - self.A @ e1)
    monkeypatch.setattr(ml.TwoLevel, "apply", bad)
    _fails(T_ml.test_vcycle_three_steps_equal_closed_form)


def test_ilu_lower_factor_off_by_a_percent(monkeypatch):
    orig = schwarz.ilu_numeric
    monkeypatch.setattr(schwarz, "ilu_numeric", lambda A, pat: (lambda LU: (1.01 * LU[0], LU[1]))(orig(A, pat)))
    _fails(T_sch.test_ilu0_tridiagonal_is_exact_lu)


def test_rate_inflow_with_the_wrong_sign(monkeypatch):
    import test_oracle_rates as T_rates
    orig = disc.Problem.__init__

    def bad(self, res):
        orig(self, res)
        if self.rate_Q is not None:
            self.rate_Q = -self.rate_Q
    monkeypatch.setattr(disc.Problem, "__init__", bad)
    _fails(T_rates.test_steady_rate_inlet_matches_the_closed_form)


def test_algorithm1_without_presmoothing(monkeypatch):
    orig = ml.MultiLevel.__init__

    def bad(self, *a, **k):
        orig(self, *a, **k)
        self.mu = 0
    monkeypatch.setattr(ml.MultiLevel, "__init__", bad)
    _fails(T_ml.test_algorithm1_two_levels_equals_vcycle)


def test_adjoint_parameter_derivative_with_the_wrong_sign(monkeypatch):
    from oracle import adjoint
    import test_oracle_adjoint as T_adj
    orig = adjoint.dF_dtheta_T
    monkeypatch.setattr(adjoint, "dF_dtheta_T", lambda *a: -orig(*a))
    _fails(T_adj.test_adjoint_gradient_matches_finite_differences, (5, 4, 2), 1)


def test_conservative_option_ignored(monkeypatch):
    import test_oracle_conservative as T_cons
    orig = disc.Problem.__init__

    def bad(self, res):
        orig(self, res)
        self.conservative = False
    monkeypatch.setattr(disc.Problem, "__init__", bad)
    _fails(T_cons.test_closed_domain_keeps_its_mass_only_in_conservative_form)


def test_upwind_option_ignored(monkeypatch):
    import test_oracle_upwind as T_up
    orig = disc.Problem.__init__

    def bad(self, res):
        orig(self, res)
        self.upwind = False
    monkeypatch.setattr(disc.Problem, "__init__", bad)
    _fails(T_up.test_upwind_telescopes_and_differs_from_the_mean)
    _fails(T_up.test_steady_flow_converges_at_first_order_from_below)
