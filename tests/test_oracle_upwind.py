"""Pins of the oracle's upstream-mobility option (Reservoir.upwind): the steady
ideal-gas flow between two fixed pressures converges at first order to the exact
profile p^2 linear in x, from below (the upstream flux p_i (p_i - p_j) exceeds the
exact (p_i^2 - p_j^2)/2 by (p_i - p_j)^2 / 2, so p^2 falls faster where p is high:
a convex profile under the chord; a downstream choice would lie above it); the
Jacobian matches central differences (with gravity too); interior fluxes
telescope; and the adjoint's flux derivative matches differences in theta."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import discretization as disc
from oracle import eos, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn


def steady_ideal_gas(n, pR=5 * syn.ATM):
    grid = syn.Grid(n, 1, 1, 100.0 / n, 1.0, 1.0)
    k = np.full(n, 1e-13)
    pL = 10 * syn.ATM
    conns = syn.dirichlet_faces(grid, k, k, k, [(0, 0, pL), (n - 1, 0, pR)])
    res = syn.Reservoir(grid, syn.Fluid(), k.copy(), k.copy(), k.copy(), np.full(n, 0.2), conns, upwind=True)
    prob = disc.Problem(res)
    prob.a, prob.b = 0.0, 0.0                    # ideal gas: Z = 1, m proportional to p
    _, _, _, _, prob.conn_m, _ = eos.eos_state(prob.conn_p, res.fluid, 0.0, 0.0)
    fac = lambda A, J: schwarz.Schwarz(A, (n, 1, 1), (4, 1, 1), 1)
    p0 = np.full(n, 7 * syn.ATM)
    p, _ = newton.newton_solve(prob, fac, p0, p0, 1e16, 1, rtol=1e-13, atol=0.0, lin_rtol=1e-12, lin_atol=0.0)
    x = (np.arange(n) + 0.5) / n
    u = pL ** 2 + (pR ** 2 - pL ** 2) * x
    return p, u, pL


def test_steady_flow_converges_at_first_order_from_below():
    errs = []
    for n in (40, 80, 160):
        p, u, pL = steady_ideal_gas(n)
        assert np.all(p ** 2 < u)
        errs.append(np.abs(p - np.sqrt(u)).max() / pL)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.1 and 1.8 < r2 < 2.1


@pytest.mark.parametrize("gravity", [0.0, 50 * 9.80665])
def test_jacobian_with_upwind_matches_central_differences(gravity):
    res = dataclasses.replace(syn.small_3d(4, 3, 4, seed=7), upwind=True, gravity=gravity)
    prob = disc.Problem(res)
    p = 4e6 + 2e6 * np.random.default_rng(3).random(res.grid.n)
    p_l, p_lm1, dt = 0.98 * p, 0.97 * p, 8640.0
    F, J = disc.residual(prob, p, p_l, p_lm1, dt, 2, want_jac=True)
    A = disc.jacobian_csr(prob.grid, J).toarray()
    n = p.size
    fd = np.zeros((n, n))
    for j in range(n):
        h = 1e-7 * p[j]                            # well inside every face's upstream choice
        e = np.zeros(n)
        e[j] = h
        fd[:, j] = (disc.residual(prob, p + e, p_l, p_lm1, dt, 2)
                    - disc.residual(prob, p - e, p_l, p_lm1, dt, 2)) / (2 * h)
    assert np.abs(A - fd).max() / np.abs(fd).max() < 1e-6


def test_upwind_telescopes_and_differs_from_the_mean():
    base = syn.small_3d(5, 4, 3, seed=2)
    p = 4e6 + 2e6 * np.random.default_rng(4).random(base.grid.n)
    up = disc.Problem(dataclasses.replace(base, upwind=True))
    F = disc.residual(up, p, 0.99 * p, 0.98 * p, 8640.0, 2)
    S = disc.storage(up, p, 0.99 * p, 0.98 * p, 8640.0, 2)
    Q = disc.connection_flux(up, p)
    assert abs(F.sum() - S.sum() - Q.sum()) < 1e-12 * np.abs(F).sum()
    Fm = disc.residual(disc.Problem(base), p, 0.99 * p, 0.98 * p, 8640.0, 2)
    assert np.abs(F - Fm).max() > 1e-6 * np.abs(Fm).max()


def test_adjoint_flux_derivative_with_upwind():
    res = dataclasses.replace(syn.small_3d(4, 3, 4, seed=6), upwind=True, gravity=50 * 9.80665)
    prob = disc.Problem(res)
    n = res.grid.n
    rng = np.random.default_rng(2)
    p = 4e6 + 2e6 * rng.random(n)
    lam = rng.standard_normal(n)
    g = oadj.dF_dtheta_T(prob, res, p, lam)
    h = 1e-6
    for i in rng.choice(n, 6, replace=False):
        e = np.zeros(n)
        e[i] = h
        fp = disc.residual(disc.Problem(oadj.perturbed(res, e)), p, 0.99 * p, p, 8640.0, 1)
        fm = disc.residual(disc.Problem(oadj.perturbed(res, -e)), p, 0.99 * p, p, 8640.0, 1)
        assert abs(lam @ (fp - fm) / (2 * h) - g[i]) <= 1e-6 * np.abs(g).max()
