"""Parity at the full 128 x 128 x 64 (1,048,576-cell) workload in the launch
configuration the benchmark times (8 x 8 x 4 subdomains, overlap 2, coarse
grid 4x coarser, FP64 and FP32 factors).

The oracle computes the residual and Jacobian of the whole grid, the ILU(0)
solves of sampled subdomains one by one, and checks properties that hold at any
size: the Galerkin projection P^T (A z - r) = 0 of the exact coarse correction
z = P A_c^{-1} P^T r, and its own residual at the GPU's implicit-step result.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import discretization as disc
from oracle import multilevel as ml
from oracle import schwarz
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev, rel_err, STENCIL

pytestmark = pytest.mark.gpu

PARTS, OVERLAP, RATIO = (8, 8, 4), 2, (4, 4, 4)


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


@pytest.fixture(scope="module")
def full():
    res = syn.config_3d_1m()
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 3, 1.0, 3.0)
    p0 = np.full(res.grid.n, res.p0)
    F, J = disc.residual(prob, p, p0, p0, res.dt, 1, want_jac=True)
    A = disc.jacobian_csr(res.grid, J)
    return res, prob, p, p0, F, J, A


def test_full_residual_and_jacobian(ras, full):
    res, prob, p, p0, F, J, A = full
    gp = ras.Problem(res)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p0), dev(p0), res.dt, 1, Fd, gp.J)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_full_ras_apply_sampled_subdomains(ras, full, prec, tol):
    res, prob, p, p0, F, J, A = full
    g = res.grid
    gp = ras.Problem(res)
    pc = ras.Precond(gp, PARTS, OVERLAP, factor_prec=prec)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(g.n, 7)
    z = torch.full((g.n,), np.nan, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    zh = host(z)
    assert np.all(np.isfinite(zh))
    boxes = schwarz.partition((g.nx, g.ny, g.nz), PARTS, OVERLAP)
    # one box of every distinct overlapped-box shape (18 or 20 cells per axis: at
    # the grid's edge or inside), with low and high edges both represented, plus
    # the two opposite corners and an interior box
    picks = {0, 91, 255}
    for ex in (0, 1):
        for ey in (0, 1):
            for ez in (0, 1):
                ix = (0 if (ey + ez) % 2 == 0 else 7) if ex else 3
                iy = (7 if (ex + ez) % 2 == 0 else 0) if ey else 4
                iz = (0 if (ex + ey) % 2 == 0 else 3) if ez else 1
                picks.add(ix + PARTS[0] * (iy + PARTS[1] * iz))
    shapes = {tuple(boxes[i].e1[a] - boxes[i].e0[a] for a in range(3)) for i in picks}
    assert len(shapes) == 8, shapes
    for i in sorted(picks):
        b = boxes[i]
        Ai = A[b.idx][:, b.idx].tocsr()
        Ai.sort_indices()
        zi = schwarz.SubdomainSolver(Ai, "ilu", 0, prec).solve(r[b.idx])
        own = b.idx[b.own]
        assert rel_err(zh[own], zi[b.own]) < tol, i


@pytest.mark.parametrize("prec,tol", [(64, 1e-9), (32, 2e-3)])
def test_full_coarse_correction_is_a_galerkin_projection(ras, full, prec, tol):
    res, prob, p, p0, F, J, A = full
    g = res.grid
    gp = ras.Problem(res)
    pc = ras.Precond(gp, PARTS, OVERLAP, factor_prec=prec, nlevels=2, coarsen=RATIO,
                     mlevel_type=4, coarse_prec=prec)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(g.n, 8)
    z = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    zh = host(z)
    P = ml.interpolation((g.nx, g.ny, g.nz), RATIO, 2)
    lhs = P.T @ (A @ zh - r)
    assert np.linalg.norm(lhs) <= tol * np.linalg.norm(P.T @ r)


def test_full_implicit_step_meets_the_newton_test(ras, full):
    res, prob, p, p0, F, J, A = full
    g = res.grid
    gp = ras.Problem(res)
    pc = ras.Precond(gp, PARTS, OVERLAP, factor_prec=32, nlevels=2, coarsen=RATIO,
                     coarse_prec=32)
    pd = dev(p0)
    out = gp.newton_step(pc, pd, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    pn = host(pd)
    # the oracle's own residual at the GPU's result satisfies Eq. equ:nonlinear_stop
    f0 = np.linalg.norm(disc.residual(prob, p0, p0, p0, res.dt, 1))
    f1 = np.linalg.norm(disc.residual(prob, pn, p0, p0, res.dt, 1))
    assert f1 <= max(1e-6 * f0, 1e-10) * 1.01
    # discrete mass balance of the step: interior fluxes telescope, so the
    # imbalance sum(storage) + sum(connection outflow) = sum(F) is bounded by
    # the residual the Newton test accepted
    S = disc.storage(prob, pn, p0, p0, res.dt, 1)
    Q = disc.connection_flux(prob, pn)
    assert abs(S.sum() + Q.sum()) <= np.sqrt(g.n) * f1 + 1e-10 * np.abs(S).sum()
