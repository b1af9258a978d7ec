"""Inexact coarse solve of the two-level preconditioners (Remark 2, Section 4):
FGMRES(30) on the Galerkin coarse operator, preconditioned by left-RAS(ILU(0))
on the coarse grid, stopped at a relative tolerance; GPU vs the oracle's
IterativeCoarse inside the same two-level combinations."""
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
    res = syn.small_3d(*dims, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    return res, J, disc.jacobian_csr(res.grid, J)


def oracle_two_level(A, dims, parts, ov, ratios, kind, rtol, ov_c=1):
    P = ml.interpolation(dims, ratios, 2)
    Ac = ml.galerkin(A, P)
    dc = ml.coarse_dims(dims, ratios)
    pc = tuple(min(p, d) for p, d in zip(parts, dc))
    M = schwarz.Schwarz(A, dims, parts, ov)
    C = ml.IterativeCoarse(Ac, dc, pc, ov_c, rtol=rtol)
    return ml.TwoLevel(A, M, P, C, kind)


CASES = [((24, 20, 12), (3, 2, 2), 1, (2, 2, 2)), ((32, 24, 16), (4, 3, 2), 2, (4, 4, 4))]


@pytest.mark.parametrize("kind", [ml.VCYCLE, ml.ADDITIVE, ml.COARSE_ONLY])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_inexact_coarse_matches_oracle(ras, kind, case):
    dims, parts, ov, ratios = CASES[case]
    res, J, A = build(dims, seed=3 + case)
    T = oracle_two_level(A, dims, parts, ov, ratios, kind, 0.2)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, mlevel_type=kind, coarse_prec=64,
                     coarse_solver=1, coarse_rtol=0.2, coarse_overlap=1)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(res.grid.n, seed)
        z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), T(r)) < 1e-8, seed


def test_tight_inexact_coarse_approaches_exact(ras):
    dims, parts, ov, ratios = CASES[0]
    res, J, A = build(dims, seed=9)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    r = dev(syn.random_vector(res.grid.n, 3))
    out = {}
    for solver in (0, 1):
        pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, coarse_prec=64,
                         coarse_solver=solver, coarse_rtol=1e-11)
        pc.factor(Jd)
        z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
        pc.apply(r, z)
        out[solver] = host(z)
    assert rel_err(out[1], out[0]) < 1e-8


def test_fgmres_with_inexact_coarse(ras):
    res = syn.small_3d(32, 32, 16, seed=13)
    g = res.grid
    gp = ras.Problem(res)
    p = dev(syn.random_pressure(res, 2, 1.0, 3.0))
    p0 = dev(np.full(g.n, res.p0))
    F = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    its = {}
    for name, kw in (("one", dict(nlevels=1)),
                     ("iter", dict(nlevels=2, coarsen=(4, 4, 4), coarse_solver=1, coarse_rtol=0.2)),
                     ("dense", dict(nlevels=2, coarsen=(4, 4, 4)))):
        pc = ras.Precond(gp, (4, 4, 2), 1, factor_prec=32, coarse_prec=32, **kw)
        pc.factor(gp.J)
        x = torch.zeros_like(F)
        out = gp.gmres_solve(gp.J, pc, -F, x, rtol=1e-6, maxit=2000)
        assert out["converged"]
        its[name] = out["iters"]
    assert its["dense"] <= its["iter"] < its["one"], its
