"""The upstream face mobility on the GPU (ras_grid.upwind) against the oracle's
(itself pinned to the first-order steady profile): residual and Jacobian with and
without gravity, the adjoint's flux derivative, and an implicit step that meets
the oracle's Newton test."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import STENCIL, dev, host, rel_err

pytestmark = pytest.mark.gpu

G = 9.80665


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


@pytest.mark.parametrize("gravity,order", [(0.0, 1), (0.0, 2), (50 * G, 2)])
def test_residual_and_jacobian_with_upwind(ras, gravity, order):
    res = dataclasses.replace(syn.small_3d(9, 7, 6, seed=5), upwind=True, gravity=gravity)
    prob = disc.Problem(res)
    rng = np.random.default_rng(6)
    p = 4e6 + 2e6 * rng.random(res.grid.n)
    p_l, p_lm1 = 0.99 * p, 0.98 * p
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, order, want_jac=True)
    gp = ras.Problem(res)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, Fd, gp.J)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


def test_grad_logk_with_upwind(ras):
    res = dataclasses.replace(syn.small_3d(9, 7, 6, seed=6), upwind=True, gravity=50 * G)
    prob = disc.Problem(res)
    rng = np.random.default_rng(7)
    p = 4e6 + 2e6 * rng.random(res.grid.n)
    lam = rng.standard_normal(res.grid.n)
    gp = ras.Problem(res)
    g = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.grad_logk(dev(p), dev(lam), g)
    assert rel_err(host(g), oadj.dF_dtheta_T(prob, res, p, lam)) < 1e-12


def test_implicit_step_with_upwind_meets_newton_test(ras):
    res = dataclasses.replace(syn.small_3d(16, 12, 10, seed=8), upwind=True)
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
    p0 = np.full(res.grid.n, res.p0)
    pd = dev(p0)
    out = gp.newton_step(pc, pd, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    f0 = np.linalg.norm(disc.residual(prob, p0, p0, p0, res.dt, 1))
    f1 = np.linalg.norm(disc.residual(prob, host(pd), p0, p0, res.dt, 1))
    assert f1 <= max(1e-6 * f0, 1e-10) * 1.01
