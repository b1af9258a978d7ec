"""ILU(k) subdomain solvers (k = 1, 2) on the GPU vs the oracle's level-of-fill
ILU(k) (Section 3.1 with the ILU(k) variants of Section 4): one-level left-RAS,
two-level V-cycle, and the paper's trend that more fill needs fewer FGMRES
iterations."""
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


CASES = [((16, 12, 8), (2, 2, 2), 1), ((20, 18, 1), (3, 2, 1), 2), ((14, 11, 9), (2, 1, 2), 0)]


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (32, 1e-5)])
def test_iluk_left_ras_matches_oracle(ras, k, case, prec, tol):
    dims, parts, ov = CASES[case]
    res, J, A = build(dims, seed=3 + case)
    M = schwarz.Schwarz(A, dims, parts, ov, ilu_k=k, prec=prec)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=prec, ilu_k=k)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(res.grid.n, seed)
        z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), M(r)) < tol, seed


def test_iluk_in_two_level_vcycle(ras):
    dims, parts, ov, ratios = (16, 12, 8), (2, 2, 2), 1, (2, 2, 2)
    res, J, A = build(dims, seed=11)
    P = ml.interpolation(dims, ratios, 2)
    M = schwarz.Schwarz(A, dims, parts, ov, ilu_k=1)
    T = ml.TwoLevel(A, M, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.VCYCLE)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, coarse_prec=64, ilu_k=1)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 5)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 1e-9


def test_fill_cuts_iterations(ras):
    """ILU(1) and ILU(2) both need fewer FGMRES iterations than ILU(0) (the paper's
    trend; between k = 1 and k = 2 the counts are close and not ordered)."""
    res = syn.small_3d(32, 32, 16, seed=13)
    g = res.grid
    gp = ras.Problem(res)
    p = dev(syn.random_pressure(res, 2, 1.0, 3.0))
    p0 = dev(np.full(g.n, res.p0))
    F = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    its = {}
    for k in (0, 1, 2):
        pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32, ilu_k=k)
        pc.factor(gp.J)
        x = torch.zeros_like(F)
        its[k] = gp.gmres_solve(gp.J, pc, -F, x, rtol=1e-6, maxit=3000)["iters"]
    assert max(its[1], its[2]) < its[0], its


def test_iluk_rejects_unsupported(ras):
    res = syn.small_3d(16, 16, 8, seed=2)
    gp = ras.Problem(res)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, ilu_k=1, ras_type=0)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, ilu_k=4)
