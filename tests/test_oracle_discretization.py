"""Pins of the oracle's CCFD / BDF residual and Jacobian (Section 2)."""
import math

import numpy as np
import pytest

from oracle import discretization as disc
from oracle import eos, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn


def small_problem(nx=6, ny=5, nz=4, seed=3):
    res = syn.small_3d(nx, ny, nz, seed=seed)
    return disc.Problem(res)


def test_flux_telescoping_mass_balance():
    """Interior fluxes cancel: sum F = sum storage + sum connection outflow."""
    prob = small_problem(7, 6, 5)
    rng = np.random.default_rng(0)
    p = syn.random_pressure(prob.res, 1)
    p_l = p * (1 + 0.01 * rng.standard_normal(p.size))
    p_lm1 = p_l * (1 + 0.01 * rng.standard_normal(p.size))
    for order in (1, 2):
        F = disc.residual(prob, p, p_l, p_lm1, 8640.0, order)
        S = disc.storage(prob, p, p_l, p_lm1, 8640.0, order)
        Q = disc.connection_flux(prob, p)
        scale = np.abs(F).sum()
        assert abs(F.sum() - S.sum() - Q.sum()) < 1e-12 * scale


@pytest.mark.parametrize("order", [1, 2])
def test_jacobian_matches_central_differences(order):
    prob = small_problem(5, 4, 3)
    p = syn.random_pressure(prob.res, 2)
    p_l = 0.97 * p
    p_lm1 = 0.95 * p
    dt = 8640.0
    F, J = disc.residual(prob, p, p_l, p_lm1, dt, order, want_jac=True)
    A = disc.jacobian_csr(prob.grid, J).toarray()
    n = p.size
    fd = np.zeros((n, n))
    for j in range(n):
        h = 1e-5 * p[j]
        e = np.zeros(n)
        e[j] = h
        fd[:, j] = (disc.residual(prob, p + e, p_l, p_lm1, dt, order)
                    - disc.residual(prob, p - e, p_l, p_lm1, dt, order)) / (2 * h)
    err = np.abs(A - fd).max() / np.abs(fd).max()
    assert err < 1e-7
    # structure: nothing outside the 7-point stencil
    assert np.all((np.abs(fd) > 1e-12 * np.abs(fd).max()) <= (A != 0))


def ideal_gas_1d(n=40, k=None, L=100.0):
    grid = syn.Grid(n, 1, 1, L / n, 1.0, 1.0)
    if k is None:
        k = np.full(n, 1e-13)
    pL, pR = 10 * syn.ATM, 1 * syn.ATM
    conns = syn.dirichlet_faces(grid, k, k, k, [(0, 0, pL), (n - 1, 0, pR)])
    fluid = syn.Fluid()
    res = syn.Reservoir(grid, fluid, k.copy(), k.copy(), k.copy(), np.full(n, 0.2), conns)
    prob = disc.Problem(res)
    prob.a, prob.b = 0.0, 0.0  # ideal gas: Z = 1
    _, _, _, _, prob.conn_m, _ = eos.eos_state(prob.conn_p, fluid, 0.0, 0.0)
    return prob, pL, pR


def _solve_steady(prob, tol=1e-13):
    n = prob.grid.n
    fac = lambda A, J: schwarz.Schwarz(A, (n, 1, 1), (4, 1, 1), 1)
    p0 = np.full(n, 5 * syn.ATM)
    p, info = newton.newton_solve(prob, fac, p0, p0, 1e16, 1, rtol=tol, atol=0.0,
                                  lin_rtol=1e-12, lin_atol=0.0)
    return p


def test_ideal_gas_steady_state_p_squared_linear():
    """Z = 1, uniform k: the exact discrete steady state has p^2 linear in x."""
    n = 40
    prob, pL, pR = ideal_gas_1d(n)
    p = _solve_steady(prob)
    x = (np.arange(n) + 0.5) / n
    u = pL ** 2 + (pR ** 2 - pL ** 2) * x
    assert np.max(np.abs(p ** 2 - u) / u) < 1e-9


def test_ideal_gas_steady_heterogeneous_series_resistance():
    """Piecewise-constant k: u = p^2 at cell centres follows the series
    resistance R(x) = int dx / k (harmonic face averaging is exact in 1D)."""
    n = 30
    rng = np.random.default_rng(5)
    k = 1e-13 * np.exp(rng.uniform(-2, 2, n))
    prob, pL, pR = ideal_gas_1d(n, k)
    p = _solve_steady(prob)
    h = prob.grid.hx
    Rc = np.concatenate([[0.0], np.cumsum(h / k)])[:-1] + 0.5 * h / k
    Rtot = np.sum(h / k)
    u = pL ** 2 - (pL ** 2 - pR ** 2) * Rc / Rtot
    assert np.max(np.abs(p ** 2 - u) / u) < 1e-9


def test_bdf2_second_order_in_time():
    """Refine dt on an ideal-gas 1D transient: BDF2 errors fall by ~4x, BDF1 by ~2x."""
    n = 16
    prob, pL, pR = ideal_gas_1d(n, L=10.0)
    fac = lambda A, J: schwarz.Schwarz(A, (n, 1, 1), (2, 1, 1), 1)
    Tend = 1500.0
    x = (np.arange(n) + 0.5) / n
    p_init = np.sqrt(pL ** 2 + (pR ** 2 - pL ** 2) * x) * (1 + 0.3 * np.sin(np.pi * x))

    def run(nsteps, bdf2=True):
        dt = Tend / nsteps
        p_l = p_init.copy()
        p_lm1 = p_l.copy()
        for s in range(nsteps):
            order = 1 if (s == 0 or not bdf2) else 2
            p_new, _ = newton.newton_solve(prob, fac, p_l, p_lm1, dt, order, rtol=1e-13,
                                           atol=0.0, lin_rtol=1e-13, lin_atol=0.0)
            p_lm1, p_l = p_l, p_new
        return p_l

    ref = run(512)
    e2 = [np.abs(run(m) - ref).max() for m in (16, 32, 64)]
    e1 = [np.abs(run(m, bdf2=False) - ref).max() for m in (16, 32, 64)]
    r2 = [e2[i] / e2[i + 1] for i in range(2)]
    r1 = [e1[i] / e1[i + 1] for i in range(2)]
    assert all(3.3 < r < 4.8 for r in r2), r2
    assert all(1.7 < r < 2.4 for r in r1), r1


def test_transmissibility_uniform_equals_kA_over_h():
    res = syn.small_3d(5, 4, 3)
    k = np.full(res.grid.n, 2e-13)
    Tx, Ty, Tz = disc.face_transmissibilities(res.grid, k, k, k)
    g = res.grid
    assert np.allclose(Tx.reshape(g.nz, g.ny, g.nx)[:, :, :-1], 2e-13 * g.hy * g.hz / g.hx, rtol=1e-15, atol=0)
    assert np.all(Tx.reshape(g.nz, g.ny, g.nx)[:, :, -1] == 0)
    assert np.allclose(Tz.reshape(g.nz, g.ny, g.nx)[:-1], 2e-13 * g.hx * g.hy / g.hz, rtol=1e-15, atol=0)


def test_bdf_terms_exact_on_polynomials_in_time():
    """Eqs. implicit-method-bdf1 / -bdf2 in closed form: BDF1 gives the exact time
    derivative of a pressure linear in time, BDF2 that of one quadratic in time,
    and the derivative terms are 1/dt and 3/(2 dt)."""
    dt, t = 7.5, 40.0
    for c0, c1, c2 in ((2.0e6, 3.0e3, 0.0), (1.0e5, -2.0e2, 5.0)):
        p = lambda s: c0 + c1 * s + c2 * s * s
        dp = c1 + 2.0 * c2 * t
        D2, d2 = disc.bdf_terms(p(t), p(t - dt), p(t - 2 * dt), dt, 2)
        assert D2 == pytest.approx(dp, rel=1e-12) and d2 == pytest.approx(1.5 / dt, rel=1e-15)
        if c2 == 0.0:
            D1, d1 = disc.bdf_terms(p(t), p(t - dt), None, dt, 1)
            assert D1 == pytest.approx(dp, rel=1e-12) and d1 == pytest.approx(1.0 / dt, rel=1e-15)
