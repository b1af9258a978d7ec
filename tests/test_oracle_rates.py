"""Pins of the oracle's fixed injection rates (the paper's Case-2 fixed injection
velocity): steady ideal-gas flow from a fixed-rate inlet to a fixed outlet
pressure matches its closed form (every face carries the inlet's p_0 Q, so
p_i^2 = p_R^2 + 2 mu p_0 Q R_i with R_i the series resistance from cell i to the
outlet, p_0 the root of p_0^2 = p_R^2 + 2 mu Q R_0 p_0), the Jacobian matches
central differences, and mass balance holds with the inflow. (GPU parity:
tests/test_gpu_physics_options.py.)"""
import dataclasses

import numpy as np
import pytest

from oracle import discretization as disc
from oracle import eos, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn


def test_steady_rate_inlet_matches_the_closed_form():
    n, L = 40, 100.0
    grid = syn.Grid(n, 1, 1, L / n, 1.0, 1.0)
    rng = np.random.default_rng(3)
    k = 1e-13 * np.exp(rng.uniform(-1, 1, n))
    pR = 1 * syn.ATM
    conns = syn.dirichlet_faces(grid, k, k, k, [(n - 1, 0, pR)])
    v = 1e-5                                       # m/s through the inlet face (1 m^2)
    Q = np.zeros(n)
    Q[0] = v * grid.hy * grid.hz
    res = syn.Reservoir(grid, syn.Fluid(), k.copy(), k.copy(), k.copy(), np.full(n, 0.2), conns, rate_Q=Q)
    prob = disc.Problem(res)
    prob.a, prob.b = 0.0, 0.0                      # ideal gas: p / Z = p
    _, _, _, _, prob.conn_m, _ = eos.eos_state(prob.conn_p, res.fluid, 0.0, 0.0)
    fac = lambda A, J: schwarz.Schwarz(A, (n, 1, 1), (4, 1, 1), 1)
    p_init = np.full(n, 2 * syn.ATM)
    p, info = newton.newton_solve(prob, fac, p_init, p_init, 1e16, 1, rtol=1e-13, atol=0.0,
                                  lin_rtol=1e-12, lin_atol=0.0)
    mu = res.fluid.mu
    # series resistances 1/T of the faces from cell i to the outlet and of the outlet connection
    Rf = 1.0 / prob.Tx[:-1]
    Rc = 1.0 / prob.conn_T[0]
    Ri = np.array([Rf[i:].sum() for i in range(n)]) + Rc
    a = mu * Q[0] * Ri[0]
    p0 = a + np.sqrt(a * a + pR * pR)
    ref = np.sqrt(pR * pR + 2 * mu * p0 * Q[0] * Ri)
    assert ref[0] > 1.5 * pR                       # the rate drives a real pressure build-up
    assert np.abs(p - ref).max() < 1e-9 * ref.max()


def test_jacobian_and_mass_balance_with_rates():
    base = syn.small_3d(4, 3, 4, seed=5)
    Q = np.zeros(base.grid.n)
    Q[[0, 5, 17]] = [1e-6, 2e-6, 5e-7]
    res = dataclasses.replace(base, rate_Q=Q)
    prob = disc.Problem(res)
    p = 4e6 + 2e6 * np.random.default_rng(1).random(res.grid.n)
    p_l, p_lm1, dt = 0.98 * p, 0.97 * p, 8640.0
    F, J = disc.residual(prob, p, p_l, p_lm1, dt, 2, want_jac=True)
    A = disc.jacobian_csr(prob.grid, J).toarray()
    n = p.size
    fd = np.zeros((n, n))
    for j in range(n):
        h = 1e-5 * p[j]
        e = np.zeros(n)
        e[j] = h
        fd[:, j] = (disc.residual(prob, p + e, p_l, p_lm1, dt, 2) - disc.residual(prob, p - e, p_l, p_lm1, dt, 2)) / (2 * h)
    assert np.abs(A - fd).max() / np.abs(fd).max() < 1e-7
    S = disc.storage(prob, p, p_l, p_lm1, dt, 2)
    out = disc.connection_flux(prob, p).sum() - disc.rate_inflow(prob, p).sum()
    assert abs(F.sum() - S.sum() - out) < 1e-12 * np.abs(F).sum()
