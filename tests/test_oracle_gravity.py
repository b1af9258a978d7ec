"""Pins of the oracle's gravity term (Eq. gover_sys, rho from Eq. equ:density):
the equilibrium of a closed column is the hydrostatic profile dp/dz = rho(p) g
(integrated independently with RK4 on the PR density), the Jacobian matches
central differences, interior fluxes still telescope, gravity = 0 is the
gravity-free model, and the adjoint's flux derivative matches differences of the
residual in log-permeability."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import discretization as disc
from oracle import eos
from paper_2007_13966_gb300 import synthetic as syn

G = 9.80665


def column(nz=30, hz=2.0, p_top=8e6, gravity=G):
    """A 1 x 1 x nz column, closed except a fixed-pressure connection on the top cell."""
    grid = syn.Grid(1, 1, nz, 10.0, 10.0, hz)
    n = grid.n
    k = np.full(n, 1e-13)
    conns = syn.Connections(np.array([0]), np.array([p_top]), np.array([1e-10]))
    res = syn.Reservoir(grid, syn.Fluid(), k, k.copy(), k.copy(), np.full(n, 0.2), conns, p0=p_top,
                        gravity=gravity)
    return res


def flux_only(prob, p):
    """Residual and Jacobian without the accumulation term (p^l = p)."""
    F, J = disc.residual(prob, p, p, p, 1.0, 1, want_jac=True)
    _, _, c, _, _, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    J["c"] = J["c"] - prob.V * prob.phi * c       # d/dp of V phi c (p - p^l)/dt at p^l = p
    return F, disc.jacobian_csr(prob.grid, J)


def density(p, fl, a, b):
    Z = eos.z_factor(np.atleast_1d(p), a, b, fl.R, fl.T)
    return float(p * fl.W / (Z[0] * fl.R * fl.T))


def test_closed_column_settles_to_the_hydrostatic_profile():
    res = column()
    prob = disc.Problem(res)
    fl = res.fluid
    a, b = prob.a, prob.b
    p = np.full(res.grid.n, res.p0)
    for _ in range(30):
        F, A = flux_only(prob, p)
        dp = np.linalg.solve(A.toarray(), -F)
        p = p + dp
        if np.abs(dp).max() < 1e-9 * p.max():
            break
    # independent: dp/dz = rho(p) g from the top cell centre, RK4 with 16 substeps per cell
    hz = res.grid.hz
    ref = [p[0]]
    q = p[0]
    h = hz / 16
    for _ in range(res.grid.nz - 1):
        for _ in range(16):
            k1 = density(q, fl, a, b) * G
            k2 = density(q + 0.5 * h * k1, fl, a, b) * G
            k3 = density(q + 0.5 * h * k2, fl, a, b) * G
            k4 = density(q + h * k3, fl, a, b) * G
            q += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        ref.append(q)
    ref = np.array(ref)
    rise = ref[-1] - ref[0]
    assert rise > 0.002 * ref[0]                # pressure grows with depth (0.43 % over 58 m)
    assert abs(p[0] - res.p0) < 1e-9 * res.p0   # no flow through the top connection
    assert np.abs(p - ref).max() < 1e-6 * rise  # second-order face rule vs the ODE


@pytest.mark.parametrize("order", [1, 2])
def test_jacobian_with_gravity_matches_central_differences(order):
    res = dataclasses.replace(syn.small_3d(4, 3, 4, seed=5), gravity=50 * G)
    prob = disc.Problem(res)
    p = 4e6 + 2e6 * np.random.default_rng(1).random(res.grid.n)
    p_l, p_lm1, dt = 0.98 * p, 0.97 * p, 8640.0
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


def test_gravity_changes_only_vertical_faces_and_telescopes():
    base = syn.small_3d(5, 4, 3, seed=2)
    p = 4e6 + 2e6 * np.random.default_rng(4).random(base.grid.n)
    F0 = disc.residual(disc.Problem(base), p, 0.99 * p, 0.98 * p, 8640.0, 2)
    Fz = disc.residual(disc.Problem(dataclasses.replace(base, gravity=0.0)), p, 0.99 * p, 0.98 * p, 8640.0, 2)
    assert np.array_equal(F0, Fz)
    prob = disc.Problem(dataclasses.replace(base, gravity=G))
    F = disc.residual(prob, p, 0.99 * p, 0.98 * p, 8640.0, 2)
    S = disc.storage(prob, p, 0.99 * p, 0.98 * p, 8640.0, 2)
    Q = disc.connection_flux(prob, p)
    assert abs(F.sum() - S.sum() - Q.sum()) < 1e-12 * np.abs(F).sum()
    flat = dataclasses.replace(base, grid=syn.Grid(5, 4, 1, base.grid.hx, base.grid.hy, base.grid.hz),
                               kx=base.kx[:20], ky=base.ky[:20], kz=base.kz[:20], phi=base.phi[:20],
                               conns=syn.Connections(np.array([0]), np.array([1e6]), np.array([1e-10])))
    q = p[:20]
    F1 = disc.residual(disc.Problem(flat), q, q, q, 8640.0, 1)
    F2 = disc.residual(disc.Problem(dataclasses.replace(flat, gravity=G)), q, q, q, 8640.0, 1)
    assert np.array_equal(F1, F2)                # one layer: no vertical face, no gravity term


def test_adjoint_flux_derivative_with_gravity():
    """(dF/dtheta)^T lambda against central differences of lambda^T F in theta."""
    res = dataclasses.replace(syn.small_3d(4, 3, 4, seed=6), gravity=50 * G)
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
        fd = lam @ (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max()
