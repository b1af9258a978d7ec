"""Right-preconditioned flexible GMRES(m), Section 3 and Remark 2.

Oracle; test infrastructure only.

Solves A x = b from x0 = 0 with a (possibly varying) right preconditioner M:
Arnoldi on w = A M v_j, classical Gram-Schmidt applied twice (CGS2), Givens
rotations on the Hessenberg matrix, x = x0 + Z y with z_j = M v_j kept
(flexible form; it equals right-preconditioned GMRES when M is fixed), restart
from the true residual every m iterations.

Stopping (Eq. equ:linear_stop): ||b - A x|| <= max(rtol ||b||, atol).
Reading: the paper prints min{.,.}; the max form is PETSc's, the paper's
platform, and the one that lets rtol act at all when atol is small.
Happy breakdown when h_{j+1,j} <= 1e-14 ||A z_j||.
"""
from __future__ import annotations

import math

import numpy as np


def fgmres(Aop, M, b, rtol=1e-6, atol=0.0, restart=30, maxit=10000, x0=None,
           history=None):
    """Returns (x, info) with info = {iters, converged, history, r0, rfinal}."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = math.sqrt(float(b @ b))
    tol = max(rtol * bnorm, atol)
    hist = [] if history is None else history
    r = b - Aop(x) if x0 is not None else b.copy()
    beta = math.sqrt(float(r @ r))
    hist.append(beta)
    it = 0
    r0 = beta
    converged = beta <= tol
    while not converged and it < maxit:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = Aop(Z[j])
            wnorm0 = math.sqrt(float(w @ w))
            # CGS2: two passes of classical Gram-Schmidt
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            hn = math.sqrt(float(w @ w))
            H[j + 1, j] = hn
            breakdown = hn <= 1e-14 * wnorm0
            if not breakdown:
                V[j + 1] = w / hn
            # previous rotations on column j
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            res = abs(g[j + 1])
            hist.append(res)
            j_end = j + 1
            if res <= tol or breakdown or it >= maxit:
                break
        # y = H^{-1} g (upper triangular back substitution)
        k = j_end
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        r = b - Aop(x)
        beta = math.sqrt(float(r @ r))
        converged = beta <= tol or (abs(g[k]) <= tol)
        if not converged and it < maxit:
            hist.append(beta)
    info = {"iters": it, "converged": converged, "history": hist, "r0": r0,
            "rfinal": beta}
    return x, info
