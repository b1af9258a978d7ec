"""Discrete adjoint on the GPU vs the oracle's (oracle/adjoint.py, itself pinned
to finite differences): J^T, the adjoint right-hand side, (dF/dtheta)^T lambda,
the full gradient through torch.autograd, and central finite differences of
the GPU's own objective on 20 random cells."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def reservoir(dims=(12, 10, 4), seed=7):
    nx, ny, nz = dims
    if nz == 1:
        return syn.lognormal_reservoir(nx, ny, 1, 30.0, 30.0, 1.0, sigma=1.0, corr=3.0,
                                       seed_k=seed, seed_phi=seed + 1)
    return syn.small_3d(nx, ny, nz, seed=seed)


def test_stencil_transpose(ras):
    res = reservoir()
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 2)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    A = disc.jacobian_csr(res.grid, J)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    JT = [torch.zeros_like(Jd[0]) for _ in range(7)]
    gp.stencil_transpose(Jd, JT)
    x = syn.random_vector(res.grid.n, 3)
    y = torch.zeros_like(Jd[0])
    gp.matvec(JT, dev(x), y)
    assert rel_err(host(y), A.T @ x) < 1e-13


def test_adjoint_rhs_and_grad_logk(ras):
    res = reservoir()
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    n = res.grid.n
    p1, p2 = syn.random_pressure(res, 4), syn.random_pressure(res, 5)
    l1, l2, dphi = (syn.random_vector(n, s) for s in (6, 7, 8))
    dt = res.dt
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda")
    gp.adjoint_rhs(dev(dphi), dev(p1), dev(l1), 2.0 / dt, dev(p2), dev(l2), -0.5 / dt, rhs)
    ref = (-dphi + (2.0 / dt) * oadj.storage_coef(prob, p1) * l1
           - (0.5 / dt) * oadj.storage_coef(prob, p2) * l2)
    assert rel_err(host(rhs), ref) < 1e-13
    gp.adjoint_rhs(None, None, None, 0.0, None, None, 0.0, rhs)
    assert float(rhs.abs().max()) == 0.0
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    gp.grad_logk(dev(p1), dev(l1), g)
    gp.grad_logk(dev(p1), dev(l1), g)                        # accumulates
    assert rel_err(host(g), 2.0 * oadj.dF_dtheta_T(prob, res, p1, l1)) < 1e-12


@pytest.mark.parametrize("dims,nsteps", [((12, 10, 4), 4), ((16, 14, 1), 3)])
def test_gradient_matches_oracle_adjoint(ras, dims, nsteps):
    from paper_2007_13966_gb300 import adjoint as gadj
    res = reservoir(dims)
    cells = oadj.producer_cells(res)
    phi_ref, grad_ref, _ = oadj.adjoint_gradient(res, nsteps, cells)
    theta = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = gadj.objective(theta, res, nsteps)
    phi.backward()
    assert abs(float(phi.detach()) - phi_ref) <= 1e-10 * phi_ref
    assert rel_err(host(theta.grad), grad_ref) < 1e-7


def test_gradient_matches_finite_differences(ras):
    """Central differences (h = 1e-6) of the GPU objective on 20 random cells. The
    bound is the differences' own error: truncation O(h^2) and rounding ~eps |phi| / h,
    about 1e-10 of the largest gradient component (measured 9e-10); 1e-8 leaves room."""
    from paper_2007_13966_gb300 import adjoint as gadj
    res = reservoir((12, 10, 4), seed=9)
    nsteps = 3
    n = res.grid.n
    theta = torch.zeros(n, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = gadj.objective(theta, res, nsteps)
    phi.backward()
    g = host(theta.grad)
    idx = np.random.default_rng(8).choice(n, 20, replace=False)
    h = 1e-6
    fd = []
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fp = float(gadj.objective(torch.as_tensor(e, device="cuda"), res, nsteps))
        fm = float(gadj.objective(torch.as_tensor(-e, device="cuda"), res, nsteps))
        fd.append((fp - fm) / (2 * h))
    err = np.abs(g[idx] - np.array(fd)).max() / np.abs(g).max()
    print("fd max relative error", err)
    assert err <= 1e-8


def test_gradient_with_two_level_solves(ras):
    """The gradient does not depend on the preconditioner: two-level V-cycle
    (right-RAS smoother on J^T) for the forward and adjoint solves."""
    from paper_2007_13966_gb300 import adjoint as gadj
    res = reservoir((16, 12, 8), seed=5)
    cells = oadj.producer_cells(res)
    _, grad_ref, _ = oadj.adjoint_gradient(res, 3, cells)
    opts = gadj.AdjointOpts(parts=(2, 2, 2), overlap=1, nlevels=2, coarsen=(2, 2, 2))
    theta = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda", requires_grad=True)
    gadj.objective(theta, res, 3, opts).backward()
    assert rel_err(host(theta.grad), grad_ref) < 1e-7
