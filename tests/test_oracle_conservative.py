"""Pins of the oracle's conservative accumulation option (Reservoir.conservative):
a closed domain keeps its discrete mass sum V phi p/Z through a converged step
(the non-conservative form of Eq. gover_sys does not: O(dt) drift), the two forms
coincide for an ideal gas (Z = 1, c = 1), and the Jacobian matches central
differences. (GPU parity: tests/test_gpu_physics_options.py.)"""
import dataclasses

import numpy as np
import pytest

from oracle import discretization as disc
from oracle import eos, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn

EMPTY = syn.Connections(np.array([], dtype=np.int32), np.array([]), np.array([]))


def mass(prob, p):
    Z = eos.eos_state(p, prob.fluid, prob.a, prob.b)[0]
    return np.sum(prob.V * prob.phi * p / Z)


def test_closed_domain_keeps_its_mass_only_in_conservative_form():
    base = dataclasses.replace(syn.small_3d(8, 6, 4, seed=3), conns=EMPTY)
    p0 = 3e6 + 3e6 * np.random.default_rng(2).random(base.grid.n)
    drift = {}
    for cons in (False, True):
        prob = disc.Problem(dataclasses.replace(base, conservative=cons))
        g = prob.grid
        fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), (2, 2, 1), 1)
        p1, info = newton.newton_solve(prob, fac, p0, p0, 10 * base.dt, 1, rtol=1e-11, atol=0.0,
                                       lin_rtol=1e-12, lin_atol=0.0)
        assert info["status"] == 0
        assert np.ptp(p1) < 1e-3 * np.ptp(p0)            # the step equalises the pressure
        drift[cons] = abs(mass(prob, p1) - mass(prob, p0)) / mass(prob, p0)
    assert drift[True] < 1e-12
    assert drift[False] > 1e-4


def test_ideal_gas_forms_coincide():
    base = syn.small_3d(5, 4, 3, seed=4)
    p = 3e6 + 3e6 * np.random.default_rng(5).random(base.grid.n)
    out = []
    for cons in (False, True):
        prob = disc.Problem(dataclasses.replace(base, conservative=cons))
        prob.a, prob.b = 0.0, 0.0
        _, _, _, _, prob.conn_m, _ = eos.eos_state(prob.conn_p, base.fluid, 0.0, 0.0)
        out.append(disc.residual(prob, p, 0.97 * p, 0.95 * p, 8640.0, 2, want_jac=True))
    (F0, J0), (F1, J1) = out
    assert np.abs(F0 - F1).max() <= 1e-12 * np.abs(F0).max()
    for s in disc.STENCIL:
        assert np.abs(J0[s] - J1[s]).max() <= 1e-12 * np.abs(J0[s]).max() + 1e-300


@pytest.mark.parametrize("order", [1, 2])
def test_conservative_jacobian_matches_central_differences(order):
    res = dataclasses.replace(syn.small_3d(4, 3, 4, seed=5), conservative=True)
    prob = disc.Problem(res)
    p = 4e6 + 2e6 * np.random.default_rng(1).random(res.grid.n)
    p_l, p_lm1, dt = 0.9 * p, 0.85 * p, 8640.0
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
    assert np.abs(A - fd).max() / np.abs(fd).max() < 1e-7
