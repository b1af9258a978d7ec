"""Parity at the full 60 x 220 x 85 (1,122,000-cell) channelised workload with
the three-level V-cycle of Algorithm 1 (4 x 11 x 5 subdomains, overlap 2;
middle level 30 x 110 x 43, overlap 1; coarsest 15 x 55 x 22), FP32 and
BF16-stored factors.

The oracle computes the residual and Jacobian of the whole grid and its own
residual at the GPU's implicit-step result (the Newton test and the discrete
mass balance hold at any size); the reduced-precision states are compared with
the GPU's FP64 form, whose arithmetic the small-grid tests pin to the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, rel_err, STENCIL

pytestmark = pytest.mark.gpu

PARTS, OVERLAP, RATIO, OVERLAP_C = (4, 11, 5), 2, (2, 2, 2), 1


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


@pytest.fixture(scope="module")
def c3():
    res = syn.channelised_reservoir()
    return res, disc.Problem(res)


def precond(ras, gp, prec, cprec):
    return ras.Precond(gp, PARTS, OVERLAP, factor_prec=prec, nlevels=3, coarsen=RATIO,
                       coarse_prec=cprec, coarse_overlap=OVERLAP_C)


def test_c3_residual_and_jacobian(ras, c3):
    res, prob = c3
    p = syn.random_pressure(res, 5, 1.0, 3.0)
    p0 = np.full(res.grid.n, res.p0)
    F, J = disc.residual(prob, p, p0, p0, res.dt, 1, want_jac=True)
    gp = ras.Problem(res)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p0), dev(p0), res.dt, 1, Fd, gp.J)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


@pytest.fixture(scope="module")
def steps(ras, c3):
    """One BDF1 step from p0 with the FP64, FP32 and BF16 forms."""
    res, prob = c3
    gp = ras.Problem(res)
    p0 = np.full(res.grid.n, res.p0)
    out = {}
    for prec, cprec in ((64, 64), (32, 32), (16, 32)):
        pc = precond(ras, gp, prec, cprec)
        pd = dev(p0)
        st = gp.newton_step(pc, pd, dev(p0), dev(p0), res.dt, 1)
        out[prec] = (st, host(pd))
        del pc
    return out


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_c3_step_meets_the_newton_test(c3, steps, prec):
    res, prob = c3
    st, pn = steps[prec]
    assert st["status"] == 0
    p0 = np.full(res.grid.n, res.p0)
    f0 = np.linalg.norm(disc.residual(prob, p0, p0, p0, res.dt, 1))
    f1 = np.linalg.norm(disc.residual(prob, pn, p0, p0, res.dt, 1))
    assert f1 <= max(1e-6 * f0, 1e-10) * 1.01
    S = disc.storage(prob, pn, p0, p0, res.dt, 1)
    Q = disc.connection_flux(prob, pn)
    assert abs(S.sum() + Q.sum()) <= np.sqrt(res.grid.n) * f1 + 1e-10 * np.abs(S).sum()


@pytest.mark.parametrize("prec", [32, 16])
def test_c3_reduced_precision_state_matches_fp64(steps, prec):
    """Mixed precision changes the Krylov path, not the Newton limit: the state
    after the step agrees with the FP64 form to the nonlinear tolerance."""
    p64 = steps[64][1]
    assert rel_err(steps[prec][1], p64) < 1e-6
