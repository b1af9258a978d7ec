"""Discrete adjoint of the implicit time loop (oracle; test infrastructure only).

The paper computes no sensitivities; this module defines, for the residual of
Section 2 (Eq. gover_sys with Eq. implicit-method-bdf1 on the first step and
Eq. implicit-method-bdf2 afterwards), the gradient of a well-pressure objective
with respect to per-cell log-permeability multipliers, by the discrete adjoint.

* Parameters: theta_i scales every permeability component of cell i,
  k_{a,i} = k0_{a,i} exp(theta_i), and the transmissibility of the cell's
  fixed-pressure connections (proportional to its permeability: half-cell well
  index and Dirichlet faces).
* Objective: Phi = sum_{l=1..L} sum_{q in cells} (p_q^l)^2.
* Adjoint, for l = L .. 1 (J_l = dF^l/dp^l at the converged p^l; s(p) = V phi c(p)):
      J_l^T lambda^l = -dPhi/dp^l + (2/dt) s(p^{l+1}) lambda^{l+1} - (1/(2 dt)) s(p^{l+2}) lambda^{l+2}
  (the two history terms are dF^{l+1}/dp^l and dF^{l+2}/dp^l of the BDF2 steps;
  terms beyond L are absent), and dPhi/dtheta = sum_l (dF^l/dtheta)^T lambda^l.
* dF/dtheta: a face flux T_f mbar (p_i - p_j) enters F_i and -F_j, and with the
  harmonic T_f = A / (h/(2 k_i) + h/(2 k_j)), dT_f/dtheta_i = T_f k_j / (k_i + k_j);
  a connection term T_q mbar (p_i - p_q) has dT_q/dtheta_i = T_q.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import discretization as disc
from . import eos
from . import newton


def perturbed(res, theta):
    """The reservoir with permeabilities (and connection transmissibilities)
    multiplied by exp(theta)."""
    from dataclasses import replace
    e = np.exp(np.asarray(theta, dtype=np.float64))
    c = res.conns
    conns = type(c)(c.cell.copy(), c.p.copy(), c.T * e[c.cell])
    return replace(res, kx=res.kx * e, ky=res.ky * e, kz=res.kz * e, conns=conns)


def _exact_precond(A, J):
    lu = spla.splu(A.tocsc())
    return lu.solve


def simulate_states(res, nsteps, rtol=1e-12, atol=0.0):
    """States p^0 .. p^L of the time loop, Newton with exact linear solves."""
    prob = disc.Problem(res)
    dt = res.dt
    p_l = np.full(prob.grid.n, res.p0)
    p_lm1 = p_l.copy()
    states = [p_l.copy()]
    for step in range(nsteps):
        order = 1 if step == 0 else 2
        p_new, info = newton.newton_solve(prob, _exact_precond, p_l, p_lm1, dt, order, rtol=rtol,
                                          atol=atol, lin_rtol=1e-14, lin_atol=0.0)
        p_lm1, p_l = p_l, p_new
        states.append(p_new.copy())
    return prob, states


def objective(states, cells):
    return float(sum(np.sum(p[cells] ** 2) for p in states[1:]))


def storage_coef(prob, p):
    """s(p) = V phi c(p)."""
    _, _, c, _, _, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    return prob.V * prob.phi * c


def dF_dtheta_T(prob, res, p, lam):
    """(dF/dtheta)^T lam at state p."""
    g = prob.grid
    Z, _, _, _, m, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    fl = prob.fluid
    rho = p * fl.W / (Z * fl.R * fl.T)
    out = np.zeros(g.n)
    for T, k, sh, dh in ((prob.Tx, res.kx, 1, 0.0), (prob.Ty, res.ky, g.nx, 0.0),
                         (prob.Tz, res.kz, g.nx * g.ny, -g.hz)):
        i = np.nonzero(T > 0)[0]
        j = i + sh
        # the face flux of the residual (gravity term included): only T_f depends on theta
        phi_ij = p[i] - p[j] - 0.5 * (rho[i] + rho[j]) * prob.gravity * dh
        mf = np.where(phi_ij >= 0, m[i], m[j]) if prob.upwind else 0.5 * (m[i] + m[j])
        flux = T[i] * mf * phi_ij
        w = (lam[i] - lam[j]) * flux / (k[i] + k[j])
        np.add.at(out, i, w * k[j])
        np.add.at(out, j, w * k[i])
    q = prob.conn_cell
    if q.size:
        np.add.at(out, q, lam[q] * disc.connection_flux(prob, p))
    return out


def adjoint_gradient(res, nsteps, cells, rtol=1e-12):
    """(Phi, dPhi/dtheta at theta = 0, the adjoint states lambda^1..lambda^L)."""
    prob, P = simulate_states(res, nsteps, rtol)
    L = nsteps
    dt = res.dt
    lam = [None] * (L + 3)
    grad = np.zeros(prob.grid.n)
    for l in range(L, 0, -1):
        order = 1 if l == 1 else 2
        p_lm2 = P[l - 2] if l >= 2 else P[l - 1]
        _, J = disc.residual(prob, P[l], P[l - 1], p_lm2, dt, order, want_jac=True)
        A = disc.jacobian_csr(prob.grid, J)
        rhs = np.zeros(prob.grid.n)
        rhs[cells] -= 2.0 * P[l][cells]
        # dF^{l+1}/dp^l = -(2/dt) s and dF^{l+2}/dp^l = (1/(2 dt)) s, with s = V phi c at
        # the newer state in Eq. gover_sys's form (c(p) D_t p) and at p^l itself in the
        # conservative form (D_t (p/Z), d(p/Z)/dp = c)
        if l + 1 <= L:
            s1 = storage_coef(prob, P[l] if prob.conservative else P[l + 1])
            rhs += (2.0 / dt) * s1 * lam[l + 1]
        if l + 2 <= L:
            s2 = storage_coef(prob, P[l] if prob.conservative else P[l + 2])
            rhs -= (0.5 / dt) * s2 * lam[l + 2]
        lam[l] = spla.spsolve(A.T.tocsc(), rhs)
        grad += dF_dtheta_T(prob, res, P[l], lam[l])
    return objective(P, cells), grad, lam[1:L + 1]


def fd_gradient(res, nsteps, cells, idx, h=1e-6, rtol=1e-12):
    """Central differences of Phi with respect to theta at the cells idx."""
    out = []
    n = res.grid.n
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        _, sp_ = simulate_states(perturbed(res, e), nsteps, rtol)
        _, sm_ = simulate_states(perturbed(res, -e), nsteps, rtol)
        out.append((objective(sp_, cells) - objective(sm_, cells)) / (2.0 * h))
    return np.array(out)


def producer_cells(res):
    """Cells of the connections at the lowest fixed pressure (the producer)."""
    c = res.conns
    return np.unique(c.cell[c.p == c.p.min()]).astype(np.int64)
