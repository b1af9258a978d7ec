"""Pins of the oracle's FGMRES (Section 3, Remark 2) and Newton/line search (Section 3)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretization as disc
from oracle import krylov, multilevel as ml, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn


def system(nx=8, ny=7, nz=3, seed=6):
    res = syn.small_3d(nx, ny, nz, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    F, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, 8640.0, 2, want_jac=True)
    return disc.jacobian_csr(res.grid, J), F, (nx, ny, nz)


def test_fgmres_identity_preconditioner_matches_dense_solve():
    A, F, dims = system()
    x, info = krylov.fgmres(lambda v: A @ v, lambda v: v, -F, rtol=1e-13, restart=200)
    ref = np.linalg.solve(A.toarray(), -F)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-12 * h[0])   # GMRES residuals never increase


def test_fgmres_ras_matches_dense_lu():
    A, F, dims = system()
    M = schwarz.Schwarz(A, dims, (2, 2, 1), 1)
    x, info = krylov.fgmres(lambda v: A @ v, M, -F, rtol=1e-13, restart=30)
    ref = np.linalg.solve(A.toarray(), -F)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    assert info["converged"]


def test_givens_estimate_equals_true_residual():
    A, F, dims = system()
    M = schwarz.Schwarz(A, dims, (2, 2, 1), 1)
    x, info = krylov.fgmres(lambda v: A @ v, M, -F, rtol=1e-6, restart=30)
    true = np.linalg.norm(-F - A @ x)
    assert abs(info["history"][-1] - true) <= 1e-8 * np.linalg.norm(F)


def test_restarted_fgmres_converges():
    A, F, dims = system(12, 10, 4)
    M = schwarz.Schwarz(A, dims, (3, 3, 2), 0)
    x, info = krylov.fgmres(lambda v: A @ v, M, -F, rtol=1e-10, restart=4, maxit=2000)
    assert info["converged"] and info["iters"] > 4
    assert np.linalg.norm(-F - A @ x) <= 1.01e-10 * np.linalg.norm(F)


def test_flexible_with_varying_preconditioner():
    """An inexact (iterative) coarse solve makes M vary; FGMRES still converges."""
    A, F, dims = system(16, 16, 1)
    P = ml.interpolation(dims, (2, 2, 1), 2)
    Ac = ml.galerkin(A, P)
    cd = ml.coarse_dims(dims, (2, 2, 1))
    coarse = ml.IterativeCoarse(Ac, cd, (2, 2, 1), 1, rtol=0.2)
    T = ml.TwoLevel(A, schwarz.Schwarz(A, dims, (2, 2, 1), 1), P, coarse)
    x, info = krylov.fgmres(lambda v: A @ v, T, -F, rtol=1e-10, restart=30)
    assert info["converged"]
    assert np.linalg.norm(-F - A @ x) <= 1.01e-10 * np.linalg.norm(F)


def test_backtrack_quadratic_step_is_exact_minimiser():
    # phi(l) = 0.5 (1 - 0.8 l)^2 * 4 -> quadratic; minimiser at l = 1.25,
    # clamped to [0.1, 0.5]; take a quadratic with minimiser inside the clamp
    phi = lambda l: 2.0 * (l - 0.3) ** 2 + 1.0
    phi0, slope, phi1 = phi(0.0), -1.2, phi(1.0)
    lam = newton.backtrack_lambda(1.0, 0.0, phi0, slope, phi1, 0.0, True)
    assert lam == pytest.approx(0.3)


def test_backtrack_cubic_step_is_exact_minimiser():
    # cubic phi with phi'(0) = slope; minimiser inside [0.1 lam, 0.5 lam]
    c3, c2, slope, c0 = 1.0, 1.0, -0.3, 2.0
    phi = lambda l: c3 * l ** 3 + c2 * l * l + slope * l + c0
    lmin = (-c2 + math.sqrt(c2 * c2 - 3 * c3 * slope)) / (3 * c3)
    lam, lam_prev = 0.5, 1.0
    new = newton.backtrack_lambda(lam, lam_prev, phi(0), slope, phi(lam), phi(lam_prev), False)
    assert 0.05 <= lmin <= 0.25
    assert new == pytest.approx(lmin, rel=1e-12)


def _problem_2d(n=24):
    res = syn.lognormal_reservoir(n, n, 1, 100.0, 100.0, 1.0, sigma=1.0, corr=4.0,
                                  seed_k=1, seed_phi=2)
    return disc.Problem(res)


def test_newton_quadratic_convergence_with_exact_solves():
    prob = _problem_2d()
    g = prob.grid
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, 1), (2, 2, 1), 10, sub="lu")
    p0 = np.full(g.n, syn.ATM)
    p, info = newton.newton_solve(prob, fac, p0, p0, 8640.0, 1, rtol=1e-12, atol=0.0,
                                  lin_rtol=1e-14, lin_atol=0.0)
    h = info["fnorm_history"]
    assert info["status"] == 0
    # once in the quadratic regime: ||F_{k+1}|| <= C ||F_k||^2 with a tame C
    ratios = [h[i + 1] / h[i] ** 2 for i in range(len(h) - 1) if h[i] < 1e-2 * h[0]]
    assert ratios and max(ratios) < 10 * min(1.0, h[0]) ** -1


def test_step_mass_balance_at_convergence():
    """Converged step: sum of storage equals minus the net connection outflow
    (interior fluxes telescope), to the Newton tolerance."""
    prob = _problem_2d(20)
    g = prob.grid
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, 1), (2, 2, 1), 1)
    p0 = np.full(g.n, syn.ATM)
    p, info = newton.newton_solve(prob, fac, p0, p0, 8640.0, 1, rtol=1e-10, atol=0.0,
                                  lin_rtol=1e-12, lin_atol=0.0)
    S = disc.storage(prob, p, p0, p0, 8640.0, 1).sum()
    Q = disc.connection_flux(prob, p).sum()
    scale = np.abs(disc.storage(prob, p, p0, p0, 8640.0, 1)).sum()
    assert abs(S + Q) <= 1e-8 * scale



@pytest.mark.parametrize("dims,parts", [((24, 24, 1), (2, 2, 1)), ((12, 12, 6), (2, 2, 1))])
def test_larger_time_steps_need_more_iterations_table_2(dims, parts):
    """Table 2's trend as a check (one-level left-RAS): one BDF1 step from the same
    state (after two 0.1-day steps) with a time step of 0.05 to 0.8 day converges
    every time, its Newton iterations do not fall and its total FGMRES iterations
    rise as the step grows."""
    res = syn.small_3d(*dims, seed=3)
    prob = disc.Problem(res)
    fac = lambda A, J: schwarz.Schwarz(A, dims, parts, 1)
    states, _ = newton.simulate(prob, fac, 2, dt=0.1 * 86400.0)
    nits, lits = [], []
    for days in (0.05, 0.1, 0.2, 0.4, 0.8):
        _, info = newton.newton_solve(prob, fac, states[-1], states[-2], days * 86400.0, 1)
        assert info["status"] == 0
        nits.append(info["newton_iters"])
        lits.append(sum(info["lin_iters"]))
    assert nits == sorted(nits), nits
    assert all(a < b for a, b in zip(lits, lits[1:])), lits
