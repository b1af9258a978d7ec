"""Inexact Newton with cubic backtracking and the BDF time loop, Sections 2-3.

Oracle; test infrastructure only.

Newton (Eq. newton_iterate): X^{k+1} = X^k + lambda^k s^k, X^0 = previous step,
J_k s^k = -F(X^k) solved by right-preconditioned (F)GMRES (Eqs. jacobian1,
jacobian), stop when ||F(X^{k+1})|| <= max(eps_r ||F(X^0)||, eps_a)
(Eq. equ:nonlinear_stop).

Line search: accept lambda when ||F(X + lambda s)|| <= (1 - alpha lambda)||F(X)||
with alpha = 1e-4 (Section 3). Otherwise backtrack on phi(lambda) =
||F(X + lambda s)||^2 / 2 (Dennis and Schnabel's cubic backtracking, the
paper's reference for the line search): the first step minimises the quadratic
through phi(0), phi'(0), phi(1); later steps the cubic through phi(0), phi'(0)
and the last two trial values; the new lambda is kept in
[0.1 lambda, 0.5 lambda]. phi'(0) = F^T J s. Reading: below lambda_min = 1e-8
the search fails. Maximum Newton iterations (not stated): 50.

Time loop (Eqs. implicit-method-bdf1, implicit-method-bdf2): BDF1 on the
first step, BDF2 afterwards, fixed dt.
"""
from __future__ import annotations

import math

import numpy as np

from . import discretization as disc
from . import krylov


def backtrack_lambda(lam, lam_prev, phi0, slope, phi_lam, phi_prev, first):
    """Next trial step length of the cubic backtracking (host scalar logic)."""
    if first:
        new = -slope / (2.0 * (phi_lam - phi0 - slope))
    else:
        t1 = phi_lam - phi0 - lam * slope
        t2 = phi_prev - phi0 - lam_prev * slope
        a = (t1 / lam ** 2 - t2 / lam_prev ** 2) / (lam - lam_prev)
        b = (-lam_prev * t1 / lam ** 2 + lam * t2 / lam_prev ** 2) / (lam - lam_prev)
        if a == 0.0:
            new = -slope / (2.0 * b)
        else:
            disc_ = b * b - 3.0 * a * slope
            if disc_ < 0.0:
                new = 0.5 * lam
            else:
                new = (-b + math.sqrt(disc_)) / (3.0 * a)
    if not np.isfinite(new):
        new = 0.5 * lam
    return min(max(new, 0.1 * lam), 0.5 * lam)


def newton_solve(prob, precond_factory, p_l, p_lm1, dt, order, rtol=1e-6, atol=1e-10,
                 maxit=50, lin_rtol=1e-6, lin_atol=1e-8, restart=30, lin_maxit=2000,
                 alpha=1e-4, lam_min=1e-8, x0=None, log=None):
    """One implicit time step. precond_factory(J_arrays) -> M (callable)."""
    X = np.array(p_l if x0 is None else x0, dtype=np.float64)
    F, J = disc.residual(prob, X, p_l, p_lm1, dt, order, want_jac=True)
    f0 = math.sqrt(float(F @ F))
    fnorm = f0
    tol = max(rtol * f0, atol)
    hist = [f0]
    lin_its = []
    lin_hists = []
    lams = []
    status = 0
    k = 0
    while fnorm > tol:
        if k >= maxit:
            status = 2
            break
        A = disc.jacobian_csr(prob.grid, J)
        M = precond_factory(A, J)
        lh = []
        s, info = krylov.fgmres(lambda v: A @ v, M, -F, rtol=lin_rtol, atol=lin_atol,
                                restart=restart, maxit=lin_maxit, history=lh)
        lin_its.append(info["iters"])
        lin_hists.append(lh)
        slope = float(F @ (A @ s))
        if slope >= 0.0:
            slope = -fnorm * fnorm
        phi0 = 0.5 * fnorm * fnorm
        lam, lam_prev, phi_prev = 1.0, 0.0, 0.0
        first = True
        while True:
            Xt = X + lam * s
            Ft, Jt = disc.residual(prob, Xt, p_l, p_lm1, dt, order, want_jac=True)
            ft = math.sqrt(float(Ft @ Ft))
            if np.isfinite(ft) and ft <= (1.0 - alpha * lam) * fnorm:
                break
            phi_t = 0.5 * ft * ft if np.isfinite(ft) else 1e300
            new = backtrack_lambda(lam, lam_prev, phi0, slope, phi_t, phi_prev, first)
            first = False
            lam_prev, phi_prev = lam, phi_t
            lam = new
            if lam < lam_min:
                status = 3
                break
        if status == 3:
            break
        lams.append(lam)
        X, F, J, fnorm = Xt, Ft, Jt, ft
        hist.append(fnorm)
        k += 1
    info = {"newton_iters": k, "fnorm_history": hist, "lin_iters": lin_its,
            "lin_histories": lin_hists, "lambdas": lams, "status": status}
    if log is not None:
        log.append(info)
    return X, info


def simulate(prob, precond_factory, nsteps, dt=None, **kw):
    """BDF1 first step, then BDF2 (fixed dt). Returns list of states and infos."""
    dt = prob.res.dt if dt is None else dt
    p_l = np.full(prob.grid.n, prob.res.p0)
    p_lm1 = p_l.copy()
    states, infos = [p_l.copy()], []
    for step in range(nsteps):
        order = 1 if step == 0 else 2
        p_new, info = newton_solve(prob, precond_factory, p_l, p_lm1, dt, order, **kw)
        infos.append(info)
        p_lm1, p_l = p_l, p_new
        states.append(p_new.copy())
    return states, infos
