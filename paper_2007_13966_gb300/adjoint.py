"""Gradient of a producer-pressure objective with respect to per-cell
log-permeability multipliers, by the discrete adjoint of the implicit time loop,
wrapped as a torch.autograd.Function.

The paper computes no sensitivities. Parameters theta scale every permeability
component of a cell, k = k0 exp(theta), and the transmissibility of the cell's
fixed-pressure connections. Objective: Phi = sum over the L steps of the squared
pressures of the producer cells (the cells of the connections at the lowest
fixed pressure). Forward: the BDF1-then-BDF2 time loop (newton_step), every
state kept as a checkpoint. Backward, for l = L .. 1, on the library's calls:
    J_l = dF^l/dp^l at p^l (residual_eval), J_l^T (ras_stencil_transpose),
    rhs = -dPhi/dp^l + (2/dt) s(p^{l+1}) lambda^{l+1} - (1/(2 dt)) s(p^{l+2}) lambda^{l+2}
          (ras_adjoint_rhs; in the conservative accumulation form the BDF weights act
          on p/Z of the older level, so both history terms take s at p^l instead),
    J_l^T lambda^l = rhs by FGMRES preconditioned by right-RAS of J_l^T
          (the transposed shape of the forward left-RAS),
    grad += (dF^l/dtheta)^T lambda^l (ras_grad_logk).
This module only sequences those calls and prepares the inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np
import torch

from . import ras


@dataclass
class AdjointOpts:
    parts: tuple = (2, 2, 1)
    overlap: int = 1
    newton_rtol: float = 1e-12
    newton_atol: float = 0.0
    lin_rtol: float = 1e-12
    adj_rtol: float = 1e-12
    restart: int = 30
    maxit: int = 4000
    nlevels: int = 1                 # 2: two-level V-cycle (forward and adjoint solves)
    coarsen: tuple = (4, 4, 4)


def scaled_reservoir(res, theta):
    """The reservoir with k -> k exp(theta) and connection T -> T exp(theta[cell])."""
    e = np.exp(np.asarray(theta, dtype=np.float64))
    c = res.conns
    conns = type(c)(c.cell.copy(), c.p.copy(), c.T * e[c.cell])
    return replace(res, kx=res.kx * e, ky=res.ky * e, kz=res.kz * e, conns=conns)


def producer_cells(res):
    c = res.conns
    return np.unique(c.cell[c.p == c.p.min()]).astype(np.int64)


def run_forward(res, theta, nsteps, opts: AdjointOpts):
    """(problem handle, states p^0..p^L on the device, objective, producer cells)."""
    r = scaled_reservoir(res, theta)
    gp = ras.Problem(r)
    pc = ras.Precond(gp, opts.parts, opts.overlap, factor_prec=64, nlevels=opts.nlevels,
                     coarsen=opts.coarsen, coarse_prec=64)
    N = r.grid.n
    p0 = torch.full((N,), r.p0, dtype=torch.float64, device="cuda")
    states = [p0.clone()]
    p_l, p_lm1 = p0.clone(), p0.clone()
    for step in range(nsteps):
        order = 1 if step == 0 else 2
        p = p_l.clone()
        out = gp.newton_step(pc, p, p_l, p_lm1, r.dt, order, rtol=opts.newton_rtol,
                             atol=opts.newton_atol, lin_rtol=opts.lin_rtol, lin_atol=0.0,
                             restart=opts.restart, lin_maxit=opts.maxit)
        fh = out["fnorm_history"]
        # below ~1e-12 ||F_0|| the residual sits at the FP64 rounding floor, where the
        # line search can no longer show a decrease: such a state is converged
        if out["status"] != 0 and not (fh and fh[-1] <= 1e-10 * fh[0]):
            raise RuntimeError(f"newton_step status {out['status']}")
        p_lm1, p_l = p_l, p
        states.append(p.clone())
    cells = torch.as_tensor(producer_cells(r), device="cuda")
    phi = sum(torch.sum(s[cells] ** 2) for s in states[1:])
    return gp, states, phi, cells


def adjoint_gradient(gp, dt, states, cells, opts: AdjointOpts, conservative=False):
    """dPhi/dtheta for the checkpointed states."""
    L = len(states) - 1
    N = states[0].numel()
    f64 = dict(dtype=torch.float64, device="cuda")
    JT = [torch.zeros(N, **f64) for _ in range(7)]
    F = torch.zeros(N, **f64)
    rhs = torch.zeros(N, **f64)
    dphi = torch.zeros(N, **f64)
    grad = torch.zeros(N, **f64)
    pcT = ras.Precond(gp, opts.parts, opts.overlap, factor_prec=64, ras_type=2,
                      nlevels=opts.nlevels, coarsen=opts.coarsen, coarse_prec=64)
    lam = [None] * (L + 3)
    for l in range(L, 0, -1):
        order = 1 if l == 1 else 2
        gp.residual_eval(states[l], states[l - 1], states[l - 2] if l >= 2 else None, dt, order,
                         F, gp.J)
        gp.stencil_transpose(gp.J, JT)
        dphi.zero_()
        dphi[cells] = 2.0 * states[l][cells]
        # dF^{l+1}/dp^l and dF^{l+2}/dp^l: s at the newer state (Eq. gover_sys's
        # c(p) D_t p) or at p^l itself (conservative form, D_t of p/Z)
        p1, l1 = (states[l] if conservative else states[l + 1], lam[l + 1]) if l + 1 <= L else (None, None)
        p2, l2 = (states[l] if conservative else states[l + 2], lam[l + 2]) if l + 2 <= L else (None, None)
        gp.adjoint_rhs(dphi, p1, l1, 2.0 / dt, p2, l2, -0.5 / dt, rhs)
        pcT.factor(JT)
        x = torch.zeros(N, **f64)
        out = gp.gmres_solve(JT, pcT, rhs, x, restart=opts.restart, maxit=opts.maxit,
                             rtol=opts.adj_rtol, atol=0.0)
        if not out["converged"] and out["rfinal"] > 1e3 * opts.adj_rtol * out["r0"]:
            raise RuntimeError("adjoint FGMRES did not converge")
        lam[l] = x
        gp.grad_logk(states[l], x, grad)
    return grad


class ProducerPressureObjective(torch.autograd.Function):
    """Phi(theta) for a reservoir template and a number of steps; backward by
    the discrete adjoint."""

    @staticmethod
    def forward(ctx, theta, res, nsteps, opts):
        th = theta.detach().to("cpu", torch.float64).numpy()
        gp, states, phi, cells = run_forward(res, th, nsteps, opts)
        ctx.saved = (gp, states, cells, res.dt, opts, bool(getattr(res, "conservative", False)))
        return phi.detach().clone()

    @staticmethod
    def backward(ctx, g):
        gp, states, cells, dt, opts, cons = ctx.saved
        grad = adjoint_gradient(gp, dt, states, cells, opts, conservative=cons)
        return g * grad, None, None, None


def objective(theta, res, nsteps, opts=None):
    return ProducerPressureObjective.apply(theta, res, nsteps, opts or AdjointOpts())
