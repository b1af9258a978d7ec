"""Two-level Schwarz on the GPU vs the oracle (Section 3.2): interpolation,
restriction R = P^T, Galerkin coarse operator, exact coarse solve (dense block
LU on the GPU, dense LU in the oracle), and the five two-level combinations."""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import multilevel as ml
from oracle import newton, schwarz
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


# (fine dims, parts, overlap, ratios): padded blocks, several blocks, multi-tile
# Gauss-Jordan (T = 192), ragged coarse cells, 2D
CASES = [
    ((16, 12, 8), (2, 2, 2), 1, (2, 2, 2)),
    ((24, 20, 12), (3, 2, 2), 2, (4, 4, 4)),
    ((40, 40, 8), (4, 4, 1), 1, (2, 2, 2)),
    ((21, 13, 10), (3, 2, 2), 1, (4, 2, 3)),
    ((32, 32, 1), (4, 4, 1), 1, (4, 4, 1)),
]


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


def oracle_two_level(A, dims, parts, ov, ratios, kind, prec=64):
    P = ml.interpolation(dims, ratios, 2)
    Ac = ml.galerkin(A, P)
    M = schwarz.Schwarz(A, dims, parts, ov, prec=prec)
    return ml.TwoLevel(A, M, P, ml.DenseCoarse(Ac), kind)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_coarse_only_correction_fp64(ras, case):
    dims, parts, ov, ratios = CASES[case]
    res, J, A = build(dims)
    T = oracle_two_level(A, dims, parts, ov, ratios, ml.COARSE_ONLY)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, mlevel_type=4, coarse_prec=64)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(res.grid.n, seed)
        z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), T(r)) < 1e-9


@pytest.mark.parametrize("kind", [ml.VCYCLE, ml.LEFT_KASKADE, ml.RIGHT_KASKADE, ml.ADDITIVE])
@pytest.mark.parametrize("case", [0, 2, 3])
def test_two_level_types_fp64(ras, kind, case):
    dims, parts, ov, ratios = CASES[case]
    res, J, A = build(dims, seed=7)
    T = oracle_two_level(A, dims, parts, ov, ratios, kind)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, mlevel_type=kind, coarse_prec=64)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 3)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 1e-9


@pytest.mark.parametrize("case", [1, 2])
def test_two_level_fp32(ras, case):
    """FP32 factors and FP32 coarse block LU against the FP64 oracle V-cycle."""
    dims, parts, ov, ratios = CASES[case]
    res, J, A = build(dims, seed=9)
    T = oracle_two_level(A, dims, parts, ov, ratios, ml.VCYCLE, prec=32)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=32, nlevels=2, coarsen=ratios, mlevel_type=0,
                     coarse_prec=32)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 4)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 5e-3


def test_two_level_newton_step_matches_oracle(ras):
    res = syn.small_3d(24, 20, 12, seed=11)
    g = res.grid
    dims, parts, ov, ratios = (g.nx, g.ny, g.nz), (3, 2, 2), 1, (2, 2, 2)
    prob = disc.Problem(res)
    P = ml.interpolation(dims, ratios, 2)

    def fac(A, J):
        M = schwarz.Schwarz(A, dims, parts, ov)
        return ml.TwoLevel(A, M, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.VCYCLE)

    p0 = np.full(g.n, res.p0)
    x_ref, info = newton.newton_solve(prob, fac, p0, p0, res.dt, 1)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, coarse_prec=64)
    p = dev(p0)
    out = gp.newton_step(pc, p, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    assert out["newton_iters"] == info["newton_iters"]
    assert out["lin_iters"] == info["lin_iters"]
    fh = np.array(out["fnorm_history"])
    ref = np.array(info["fnorm_history"])
    # 1e-9 relative, with the FP64 noise floor of ||F|| (~1e-13 ||F0||) allowed
    assert np.all(np.abs(fh - ref) <= 1e-9 * ref + 1e-12 * ref[0])
    assert rel_err(host(p), x_ref) < 1e-10


def test_two_level_fewer_iterations_than_one_level(ras):
    """The paper's qualitative claim (Tables 8-10): the coarse level cuts FGMRES
    iterations at a fixed number of subdomains."""
    res = syn.small_3d(32, 32, 16, seed=13)
    g = res.grid
    gp = ras.Problem(res)
    p = dev(syn.random_pressure(res, 2, 1.0, 3.0))
    p0 = dev(np.full(g.n, res.p0))
    F = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    its = {}
    for nl in (1, 2):
        pc = ras.Precond(gp, (4, 4, 2), 1, factor_prec=32, nlevels=nl, coarsen=(4, 4, 4),
                         coarse_prec=32)
        pc.factor(gp.J)
        x = torch.zeros_like(F)
        its[nl] = gp.gmres_solve(gp.J, pc, -F, x, rtol=1e-6, maxit=2000)["iters"]
    assert its[2] < its[1]
