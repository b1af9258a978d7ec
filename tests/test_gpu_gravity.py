"""The gravity term on the GPU (Eq. gover_sys's rho g grad h, rho of Eq.
equ:density) against the oracle's (itself pinned to the hydrostatic profile):
residual and Jacobian, the adjoint's flux derivative, and an implicit step driven
by gravity alone that meets the oracle's Newton test."""
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


def heavy(seed=5, dims=(9, 7, 6), g=50 * G):
    return dataclasses.replace(syn.small_3d(*dims, seed=seed), gravity=g)


@pytest.mark.parametrize("order", [1, 2])
def test_residual_and_jacobian_with_gravity(ras, order):
    res = heavy()
    prob = disc.Problem(res)
    rng = np.random.default_rng(3)
    p = 4e6 + 2e6 * rng.random(res.grid.n)
    p_l, p_lm1 = 0.99 * p, 0.98 * p
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, order, want_jac=True)
    gp = ras.Problem(res)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, Fd, gp.J)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


def test_grad_logk_with_gravity(ras):
    res = heavy(seed=6)
    prob = disc.Problem(res)
    rng = np.random.default_rng(4)
    p = 4e6 + 2e6 * rng.random(res.grid.n)
    lam = rng.standard_normal(res.grid.n)
    gp = ras.Problem(res)
    g = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.grad_logk(dev(p), dev(lam), g)
    assert rel_err(host(g), oadj.dF_dtheta_T(prob, res, p, lam)) < 1e-12


def test_implicit_step_with_gravity_meets_newton_test(ras):
    """A reservoir at a uniform 5 MPa, closed but for one weak connection at that
    pressure: gravity alone drives the step, and the deeper layers gain pressure."""
    base = syn.small_3d(16, 12, 10, seed=8)
    p_init = 5e6
    conns = syn.Connections(np.array([0]), np.array([p_init]), np.array([1e-12]))
    res = dataclasses.replace(base, gravity=G, p0=p_init, conns=conns)
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
    p0 = np.full(res.grid.n, p_init)
    pd = dev(p0)
    out = gp.newton_step(pc, pd, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    f0 = np.linalg.norm(disc.residual(prob, p0, p0, p0, res.dt, 1))
    f1 = np.linalg.norm(disc.residual(prob, host(pd), p0, p0, res.dt, 1))
    assert f0 > 0 and f1 <= max(1e-6 * f0, 1e-10) * 1.01
    layer = 16 * 12
    top, bottom = host(pd)[:layer], host(pd)[-layer:]
    assert bottom.mean() > p_init > top.mean()
