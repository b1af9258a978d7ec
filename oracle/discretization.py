"""CCFD (two-point flux) discretisation and BDF1/BDF2 residual, Section 2.

Oracle; test infrastructure only.

Residual of cell i (Eq. gover_sys integrated over the cell, times its volume V,
time derivative by Eq. implicit-method-bdf1 / implicit-method-bdf2):

    F_i = V phi_i c(p_i) D_t p_i + sum_faces T_f mbar_f (p_i - p_j - rhobar_f g (h_i - h_j))
          + sum_conns T_q mbar_q (p_i - p_q)

with c(p) = (p/Z)(1/p - Z'/Z) evaluated at the new level, m(p) = p / (mu Z),
D_t p = (p - p^l)/dt (BDF1) or (3p - 4p^l + p^{l-1})/(2 dt) (BDF2), and the gravity
term of Eq. gover_sys: rho(p) = p W / (Z R T) (Eq. equ:density), h the depth of the
cell centre, g = Reservoir.gravity along the z axis with depth increasing with the z
index (h_j - h_i = hz across a +z face; x and y faces are level). gravity = 0 is the
gravity-free model.

Readings (the paper defers CCFD details to its references):
* geometric face transmissibility T_f = A_f / (h/(2 k_i) + h/(2 k_j)) (harmonic);
* mbar_f = (m_i + m_j)/2 (arithmetic mean of the two cells);
* wells and Dirichlet faces are fixed-pressure connections with a half-cell
  transmissibility and mbar = (m_i + m(p_q))/2, at the depth of their cell (no
  gravity term); faces without one are no-flow;
* rhobar_f = (rho_i + rho_j)/2 (arithmetic mean, like mbar_f);
* Reservoir.upwind = True replaces mbar_f by the mobility of the upstream cell, the
  one the face potential points away from (i if p_i - p_j - rhobar g (h_i - h_j) >= 0,
  else j), for faces and connections alike (a fixed pressure upstream: m(p_q)); the
  density in the gravity term stays the mean;
* fixed injection rates (the paper's Case-2 alternative to a fixed injection pressure): a
  Darcy velocity v into the domain through boundary faces of total area A of a cell
  carries (p/Z) v A of the equation's transported quantity (Eq. gover_sys divided by
  W / (RT)), the cell's own p/Z for the injected gas: F_i -= mu m(p_i) Q_i with
  Q_i = v A (Reservoir.rate_Q, m^3/s per cell; positive into the cell);
* Reservoir.conservative = True takes the accumulation in conservative form,
  V phi D_t (p/Z) (the time derivative of Eq. mass conservation's phi rho, divided by
  W / (RT)), instead of Eq. gover_sys's V phi c(p) D_t p; the two agree for an ideal
  gas (Z = 1) and differ at O(dt) otherwise; the conservative form keeps the discrete
  mass of a closed domain exactly.
The source term -qRT/W of Eq. gover_sys is carried by the connections.

Jacobian storage: seven arrays (centre, -x, +x, -y, +y, -z, +z) of length N,
J[s][i] = dF_i / dp_{neighbour s of i}, zero where the neighbour is absent.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import eos

STENCIL = ("c", "-x", "+x", "-y", "+y", "-z", "+z")


def face_transmissibilities(grid, kx, ky, kz):
    """Harmonic-average geometric transmissibility of every +x/+y/+z face.

    Tx[i] joins cell i to cell i+1 (0 on the last x layer), likewise Ty, Tz.
    """
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    K = [np.asarray(k, dtype=np.float64).reshape(nz, ny, nx) for k in (kx, ky, kz)]
    hx, hy, hz = grid.hx, grid.hy, grid.hz
    Tx = np.zeros((nz, ny, nx))
    Ty = np.zeros((nz, ny, nx))
    Tz = np.zeros((nz, ny, nx))
    Ax, Ay, Az = hy * hz, hx * hz, hx * hy
    Tx[:, :, :-1] = Ax / (hx / (2 * K[0][:, :, :-1]) + hx / (2 * K[0][:, :, 1:]))
    Ty[:, :-1, :] = Ay / (hy / (2 * K[1][:, :-1, :]) + hy / (2 * K[1][:, 1:, :]))
    Tz[:-1, :, :] = Az / (hz / (2 * K[2][:-1, :, :]) + hz / (2 * K[2][1:, :, :]))
    return Tx.reshape(-1), Ty.reshape(-1), Tz.reshape(-1)


class Problem:
    """A reservoir with its static discretisation data."""

    def __init__(self, res):
        self.res = res
        self.grid = res.grid
        self.gravity = float(getattr(res, "gravity", 0.0))
        self.upwind = bool(getattr(res, "upwind", False))
        self.conservative = bool(getattr(res, "conservative", False))
        rq = getattr(res, "rate_Q", None)
        self.rate_Q = None if rq is None else np.asarray(rq, dtype=np.float64)
        self.fluid = res.fluid
        self.a, self.b = eos.pr_constants(res.fluid)
        self.Tx, self.Ty, self.Tz = face_transmissibilities(res.grid, res.kx, res.ky, res.kz)
        g = res.grid
        self.V = g.hx * g.hy * g.hz
        self.phi = np.asarray(res.phi, dtype=np.float64)
        self.conn_cell = res.conns.cell.astype(np.int64)
        self.conn_p = res.conns.p
        self.conn_T = res.conns.T
        _, _, _, _, self.conn_m, _ = eos.eos_state(self.conn_p, self.fluid, self.a, self.b)

    def _shifts(self):
        g = self.grid
        return (1, g.nx, g.nx * g.ny)


def bdf_terms(p, p_l, p_lm1, dt, order):
    """(D_t p, dD_t/dp) of Eq. implicit-method-bdf1 (order 1) or -bdf2 (order 2)."""
    if order == 1:
        return (p - p_l) / dt, 1.0 / dt
    return (3.0 * p - 4.0 * p_l + p_lm1) / (2.0 * dt), 1.5 / dt


def residual(prob: Problem, p, p_l, p_lm1, dt, order, want_jac=False):
    """F(p) and, optionally, the seven Jacobian arrays."""
    g = prob.grid
    N = g.n
    p = np.asarray(p, dtype=np.float64)
    Z, _, c, dc, m, dm = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    fl = prob.fluid
    rho = p * fl.W / (Z * fl.R * fl.T)         # Eq. equ:density
    drho = fl.W * c / (fl.R * fl.T)             # d rho / dp = (W / RT)(1/Z - p Z'/Z^2)
    Dt, dDt = bdf_terms(p, p_l, p_lm1, dt, order)
    if prob.conservative:
        # D_t of P = p/Z with the same BDF weights; dP/dp = c
        P = lambda q: q / eos.eos_state(q, prob.fluid, prob.a, prob.b)[0]
        DtP, _ = bdf_terms(p / Z, P(p_l), P(p_lm1) if order == 2 else None, dt, order)
        F = prob.V * prob.phi * DtP
        Jc = prob.V * prob.phi * c * dDt
    else:
        F = prob.V * prob.phi * c * Dt
        Jc = prob.V * prob.phi * (dc * Dt + c * dDt)
    J = {s: np.zeros(N) for s in STENCIL}
    # interior faces, one axis at a time (+ side of cell i joins i and i+shift)
    for T, sh, minus, plus, dh in ((prob.Tx, 1, "-x", "+x", 0.0),
                                   (prob.Ty, g.nx, "-y", "+y", 0.0),
                                   (prob.Tz, g.nx * g.ny, "-z", "+z", -g.hz)):
        i = np.nonzero(T > 0)[0]
        j = i + sh
        gdh = prob.gravity * dh                  # g (h_i - h_j)
        phi_ij = p[i] - p[j] - 0.5 * (rho[i] + rho[j]) * gdh
        if prob.upwind:
            wi = (phi_ij >= 0).astype(np.float64)  # weight of cell i in the face mobility
        else:
            wi = np.full(i.size, 0.5)
        wj = 1.0 - wi
        mf = wi * m[i] + wj * m[j] if prob.upwind else 0.5 * (m[i] + m[j])
        flux = T[i] * mf * phi_ij
        np.add.at(F, i, flux)
        np.add.at(F, j, -flux)
        # d flux / d p_i and d flux / d p_j
        dfi = T[i] * (wi * dm[i] * phi_ij + mf * (1.0 - 0.5 * drho[i] * gdh))
        dfj = T[i] * (wj * dm[j] * phi_ij + mf * (-1.0 - 0.5 * drho[j] * gdh))
        np.add.at(Jc, i, dfi)
        np.add.at(Jc, j, -dfj)
        J[plus][i] += dfj
        J[minus][j] += -dfi
    # fixed-pressure connections (wells, Dirichlet faces)
    q = prob.conn_cell
    if q.size:
        dp = p[q] - prob.conn_p
        if prob.upwind:
            wq = (dp >= 0).astype(np.float64)
            mf = wq * m[q] + (1.0 - wq) * prob.conn_m
        else:
            wq = np.full(q.size, 0.5)
            mf = 0.5 * (m[q] + prob.conn_m)
        np.add.at(F, q, prob.conn_T * mf * dp)
        np.add.at(Jc, q, prob.conn_T * (wq * dm[q] * dp + mf))
    # fixed injection rates: the cell's p/Z = mu m enters with the Darcy volume rate
    if prob.rate_Q is not None:
        mu = prob.fluid.mu
        F -= mu * m * prob.rate_Q
        Jc -= mu * dm * prob.rate_Q
    J["c"] = Jc
    if want_jac:
        return F, J
    return F


def jacobian_csr(grid, J):
    """Assemble the seven stencil arrays into a scipy CSR matrix."""
    N = grid.n
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    idx = np.arange(N)
    ii = idx % nx
    jj = (idx // nx) % ny
    kk = idx // (nx * ny)
    rows, cols, vals = [idx], [idx], [J["c"]]
    for s, sh, ok in (("-x", -1, ii > 0), ("+x", 1, ii < nx - 1),
                      ("-y", -nx, jj > 0), ("+y", nx, jj < ny - 1),
                      ("-z", -nx * ny, kk > 0), ("+z", nx * ny, kk < nz - 1)):
        rows.append(idx[ok])
        cols.append(idx[ok] + sh)
        vals.append(J[s][ok])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sort_indices()
    return A


def stencil_matvec(grid, J, x):
    """y = J x with the seven stencil arrays (plain definition)."""
    return jacobian_csr(grid, J) @ x


def storage(prob: Problem, p, p_l, p_lm1, dt, order):
    """The accumulation part of each cell: V phi c D_t p, or V phi D_t (p/Z) in the
    conservative form."""
    Z, _, c, _, _, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    if prob.conservative:
        P = lambda q: q / eos.eos_state(q, prob.fluid, prob.a, prob.b)[0]
        DtP, _ = bdf_terms(p / Z, P(p_l), P(p_lm1) if order == 2 else None, dt, order)
        return prob.V * prob.phi * DtP
    Dt, _ = bdf_terms(p, p_l, p_lm1, dt, order)
    return prob.V * prob.phi * c * Dt


def connection_flux(prob: Problem, p):
    """Per-connection outflow T m_f (p_i - p_q) (positive out of the cell)."""
    _, _, _, _, m, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    q = prob.conn_cell
    dp = p[q] - prob.conn_p
    mf = np.where(dp >= 0, m[q], prob.conn_m) if prob.upwind else 0.5 * (m[q] + prob.conn_m)
    return prob.conn_T * mf * dp


def rate_inflow(prob: Problem, p):
    """Per-cell inflow mu m(p) Q of the fixed injection rates (zero without them)."""
    if prob.rate_Q is None:
        return np.zeros(prob.grid.n)
    _, _, _, _, m, _ = eos.eos_state(p, prob.fluid, prob.a, prob.b)
    return prob.fluid.mu * m * prob.rate_Q
