"""Classical additive Schwarz (Eq. equ:as-class) and right-RAS (Eq. equ:as-right)
on the GPU vs the oracle: box solutions summed over the overlap (R_i^delta)^T,
right-RAS restricting the input to owned cells (R_i^0)."""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import multilevel as ml
from oracle import schwarz
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


def build(dims, seed=5):
    nx, ny, nz = dims
    if nz == 1:
        res = syn.lognormal_reservoir(nx, ny, 1, 50.0, 50.0, 1.0, sigma=1.0, corr=4.0,
                                      seed_k=seed, seed_phi=seed + 1)
    else:
        res = syn.small_3d(nx, ny, nz, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    return res, J, disc.jacobian_csr(res.grid, J)


# (dims, parts, overlap): several boxes per axis, an overlap wider than a part
# (three boxes cover some cells), 2D
CASES = [((24, 20, 12), (3, 2, 2), 1), ((20, 16, 10), (4, 4, 2), 3), ((32, 28, 1), (3, 3, 1), 2)]


@pytest.mark.parametrize("kind", [schwarz.AS, schwarz.RIGHT_RAS])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_kind_matches_oracle(ras, kind, case, prec, tol):
    dims, parts, ov = CASES[case]
    res, J, A = build(dims, seed=3 + case)
    M = schwarz.Schwarz(A, dims, parts, ov, kind=kind, prec=prec)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=prec, ras_type=kind)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(res.grid.n, seed)
        z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), M(r)) < tol, seed


def test_kinds_agree_without_overlap(ras):
    """delta = 0: AS = left-RAS = right-RAS = block Jacobi."""
    dims, parts = (24, 20, 12), (3, 2, 2)
    res, J, A = build(dims, seed=8)
    gp = ras.Problem(res)
    r = dev(syn.random_vector(res.grid.n, 4))
    outs = []
    for kind in (0, 1, 2):
        pc = ras.Precond(gp, parts, 0, ras_type=kind)
        pc.factor(j_to_dev(J))
        z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
        pc.apply(r, z)
        outs.append(host(z))
    assert rel_err(outs[0], outs[1]) < 1e-14
    assert rel_err(outs[2], outs[1]) < 1e-14


def test_as_overlap_sum_is_deterministic(ras):
    dims, parts, ov = CASES[1]
    res, J, A = build(dims, seed=9)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=32, ras_type=schwarz.AS)
    pc.factor(j_to_dev(J))
    r = dev(syn.random_vector(res.grid.n, 6))
    zs = []
    for _ in range(3):
        z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
        pc.apply(r, z)
        zs.append(host(z))
    assert np.array_equal(zs[0], zs[1]) and np.array_equal(zs[0], zs[2])


def test_two_level_vcycle_with_as_smoother(ras):
    dims, parts, ov, ratios = (24, 20, 12), (3, 2, 2), 1, (2, 2, 2)
    res, J, A = build(dims, seed=11)
    P = ml.interpolation(dims, ratios, 2)
    M = schwarz.Schwarz(A, dims, parts, ov, kind=schwarz.AS)
    T = ml.TwoLevel(A, M, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.VCYCLE)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, coarse_prec=64,
                     ras_type=schwarz.AS)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 5)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 1e-9


@pytest.mark.parametrize("kind", [schwarz.AS, schwarz.RIGHT_RAS])
def test_fgmres_converges_with_kind(ras, kind):
    res = syn.small_3d(32, 32, 16, seed=13)
    g = res.grid
    gp = ras.Problem(res)
    p = dev(syn.random_pressure(res, 2, 1.0, 3.0))
    p0 = dev(np.full(g.n, res.p0))
    F = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    pc = ras.Precond(gp, (4, 4, 2), 1, factor_prec=32, ras_type=kind)
    pc.factor(gp.J)
    x = torch.zeros_like(F)
    out = gp.gmres_solve(gp.J, pc, -F, x, rtol=1e-6, maxit=2000)
    assert out["converged"]
    Ax = torch.zeros_like(F)
    gp.matvec(gp.J, x, Ax)
    assert float(torch.linalg.norm(Ax + F)) <= 1.01e-6 * float(torch.linalg.norm(F))
