"""Multilevel Schwarz preconditioners, Section 3.2 (oracle; test infrastructure only).

* Coarse mesh (Fig. 2): geometry preserving; coarse cell I covers fine cells
  [rI, min(rI + r, n)) per axis and its centre is the centre of that range, so
  coarse and fine centres do not coincide.
* Interpolation I_{j-1}^j: first order (nearest centre, Eq. equ:inter-frist),
  second order (tensor-product linear, Eq. equ:inter-second) and third order
  (cubic convolution with a = -1/2, Eq. equ:inter-third), built per axis and
  combined by Kronecker products.
  Readings: beyond the outermost coarse centres the linear weights extrapolate
  by a constant (all weight on the boundary coarse cell); the cubic kernel's
  stencil indices are clamped to the coarse range; ties in nearest-neighbour
  go to the lower index; W(0) = 1 and W(+-1) = W(+-2) = 0 by continuity.
* Restriction I_j^{j-1}: the live text never defines it (only commented-out
  weights survive); reading: R = P^T.
* Coarse operator A_{h_{j-1}}: not stated; reading: Galerkin R A P.
* Two-level preconditioners with mu = nu = 1: V-cycle (Eq. equ:v-cycle, the
  three-step form of Eq. two_level_preconditioner), left-Kaskade
  (Eq. equ:left-Kas), right-Kaskade (Eq. equ:right-Kas), additive
  (Eq. equ:two-additive), coarse-only (Eq. equ:coarse-level).
* L >= 3 levels: Algorithm 1 (MG V-cycle with Schwarz-preconditioned
  Richardson smoothing, zero initial guess on every coarser level).
* Coarsest solve: dense LU (exact), or GMRES preconditioned by one-level
  Schwarz at a relative tolerance (Remark 2).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import krylov, schwarz

VCYCLE, LEFT_KASKADE, RIGHT_KASKADE, ADDITIVE, COARSE_ONLY = 0, 1, 2, 3, 4


def coarse_size(n: int, r: int) -> int:
    return (n + r - 1) // r if n > 1 else 1


def coarse_centres(n: int, r: int):
    nc = coarse_size(n, r)
    return np.array([(r * I + min(r * I + r, n)) / 2.0 for I in range(nc)])


def keys_w(s: float) -> float:
    """Cubic-convolution weight W(s), a = -1/2 (Eq. equ:inter-third)."""
    s = abs(s)
    if s < 1.0:
        return 1.5 * s ** 3 - 2.5 * s ** 2 + 1.0
    if s < 2.0:
        return -0.5 * s ** 3 + 2.5 * s ** 2 - 4.0 * s + 2.0
    return 0.0


def interp_1d(n: int, r: int, order: int) -> np.ndarray:
    """Dense n x nc interpolation matrix along one axis."""
    if n == 1:
        return np.ones((1, 1))
    nc = coarse_size(n, r)
    xc = coarse_centres(n, r)
    P = np.zeros((n, nc))
    for i in range(n):
        x = i + 0.5
        if order == 1:
            d = np.abs(xc - x)
            P[i, int(np.argmin(d))] = 1.0   # argmin returns the lower index on ties
            continue
        # bracketing coarse centres xc[I0] <= x < xc[I0+1]
        I0 = int(np.searchsorted(xc, x, side="right")) - 1
        if order == 2:
            if I0 < 0:
                P[i, 0] = 1.0
            elif I0 >= nc - 1:
                P[i, nc - 1] = 1.0
            else:
                t = (x - xc[I0]) / (xc[I0 + 1] - xc[I0])
                P[i, I0] += 1.0 - t
                P[i, I0 + 1] += t
            continue
        # order 3: 4 nodes I0-1 .. I0+2, spacing r (uniform coarse centres)
        if nc == 1:
            P[i, 0] = 1.0
            continue
        base = int(np.floor((x - xc[0]) / r))   # node lattice xc[0] + J r
        for l in range(-1, 3):
            J = base + l
            s = (x - (xc[0] + J * r)) / r
            w = keys_w(s)
            P[i, min(max(J, 0), nc - 1)] += w
    return P


def interpolation(grid_dims, ratios, order) -> sp.csr_matrix:
    """I_{j-1}^j for a grid (nx, ny, nz) with per-axis ratios; x fastest."""
    Px = sp.csr_matrix(interp_1d(grid_dims[0], ratios[0], order))
    Py = sp.csr_matrix(interp_1d(grid_dims[1], ratios[1], order))
    Pz = sp.csr_matrix(interp_1d(grid_dims[2], ratios[2], order))
    return sp.kron(sp.kron(Pz, Py), Px).tocsr()


def coarse_dims(grid_dims, ratios):
    return tuple(coarse_size(grid_dims[a], ratios[a]) for a in range(3))


class DenseCoarse:
    """Exact coarsest solve by dense LU (no pivoting needed in exact arithmetic;
    partial pivoting is used here since only A_c^{-1} matters)."""

    def __init__(self, Ac):
        self.lu = sla.lu_factor(Ac.toarray())

    def __call__(self, r):
        return sla.lu_solve(self.lu, r)


class IterativeCoarse:
    """Coarsest solve by one-level-Schwarz-preconditioned GMRES (Remark 2)."""

    def __init__(self, Ac, dims, parts, overlap, rtol=0.2, restart=30, maxit=200,
                 kind=schwarz.LEFT_RAS, sub="ilu", ilu_k=0):
        self.Ac = Ac
        self.M = schwarz.Schwarz(Ac, dims, parts, overlap, kind, sub, ilu_k)
        self.rtol, self.restart, self.maxit = rtol, restart, maxit

    def __call__(self, r):
        x, _ = krylov.fgmres(lambda v: self.Ac @ v, self.M, r, rtol=self.rtol,
                             atol=0.0, restart=self.restart, maxit=self.maxit)
        return x


class TwoLevel:
    """Two-level preconditioner of the given type (mu = nu = 1)."""

    def __init__(self, A, M_fine, P, coarse_solve, kind=VCYCLE):
        self.A, self.M, self.P = A, M_fine, P
        self.R = P.T.tocsr()
        self.C = coarse_solve
        self.kind = kind

    def coarse(self, r):
        return self.P @ self.C(self.R @ r)

    def apply(self, r):
        A, M = self.A, self.M
        if self.kind == VCYCLE:               # Eq. equ:v-cycle
            e1 = M(r)
            e2 = e1 + self.coarse(r - A @ e1)
            return e2 + M(r - A @ e2)
        if self.kind == LEFT_KASKADE:         # Eq. equ:left-Kas
            c = self.coarse(r)
            return c + M(r) - M(A @ c)
        if self.kind == RIGHT_KASKADE:        # Eq. equ:right-Kas
            e = M(r)
            return e + self.coarse(r) - self.coarse(A @ e)
        if self.kind == ADDITIVE:             # Eq. equ:two-additive
            return self.coarse(r) + M(r)
        if self.kind == COARSE_ONLY:          # Eq. equ:coarse-level
            return self.coarse(r)
        raise ValueError(self.kind)

    def __call__(self, r):
        return self.apply(r)


class MultiLevel:
    """Algorithm 1 (MG V-cycle) over L levels with Schwarz-Richardson smoothing.

    levels[j] = (A_j, M_j) for j = 1..L-1 (fine is L-1), Ps[j] interpolates from
    level j-1 to level j, coarsest solve `coarse` on level 0.
    """

    def __init__(self, As, Ms, Ps, coarse, mu=1, nu=1):
        self.As, self.Ms, self.Ps, self.coarse = As, Ms, Ps, coarse
        self.mu, self.nu = mu, nu

    def mg(self, b, j, x):
        if j == 0:
            return self.coarse(b)
        A, M = self.As[j], self.Ms[j]
        for _ in range(self.mu):             # presmoothing: x += M (b - A x)
            x = x + M(b - A @ x)
        bc = self.Ps[j].T @ (b - A @ x)       # residual restriction
        xc = self.mg(bc, j - 1, np.zeros(bc.size))
        x = x + self.Ps[j] @ xc               # correction interpolation
        for _ in range(self.nu):             # postsmoothing
            x = x + M(b - A @ x)
        return x

    def __call__(self, r):
        L = len(self.As) - 1
        return self.mg(r, L, np.zeros_like(r))


def galerkin(A, P):
    """A_c = P^T A P (reading: Galerkin coarse operator)."""
    Ac = (P.T @ A @ P).tocsr()
    Ac.sort_indices()
    return Ac
