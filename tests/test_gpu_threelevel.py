"""Three-level Schwarz on the GPU vs the oracle (Section 3.2, Algorithm 1):
Galerkin operators A_1 = P_1^T A P_1 and A_0 = P_0^T A_1 P_0, RAS(ILU(0))
Richardson smoothing on the fine and middle levels (the middle-level ILU(0) on
A_1's nonzero pattern, overlap delta_c), exact coarsest solve."""
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


# (fine dims, parts, overlap, coarse overlap, ratios): middle-level boxes
# thinner than the 5-cell reach of A_1 (natural order differs from offset
# order), several shapes, ragged coarse cells, 2D, odd sizes, delta_c = 0 and 2
CASES = [
    ((24, 20, 16), (2, 2, 2), 1, 1, (2, 2, 2)),
    ((32, 28, 12), (3, 2, 2), 2, 1, (2, 2, 2)),
    ((40, 36, 1), (3, 3, 1), 1, 1, (2, 2, 1)),
    ((25, 19, 11), (2, 2, 1), 1, 2, (2, 2, 2)),
    ((30, 24, 16), (2, 3, 2), 1, 0, (2, 2, 2)),
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


def oracle_three_level(A, dims, parts, ov, ov_c, ratios, prec=64):
    P1 = ml.interpolation(dims, ratios, 2)
    A1 = ml.galerkin(A, P1)
    d1 = ml.coarse_dims(dims, ratios)
    P0 = ml.interpolation(d1, ratios, 2)
    A0 = ml.galerkin(A1, P0)
    M2 = schwarz.Schwarz(A, dims, parts, ov, prec=prec)
    M1 = schwarz.Schwarz(A1, d1, parts, ov_c, prec=prec)
    return ml.MultiLevel([A0, A1, A], [None, M1, M2], [None, P0, P1], ml.DenseCoarse(A0))


def gpu_three_level(ras, res, parts, ov, ov_c, ratios, prec=64, cprec=64):
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=prec, nlevels=3, coarsen=ratios, mlevel_type=0,
                     coarse_prec=cprec, coarse_overlap=ov_c)
    return gp, pc


@pytest.mark.parametrize("case", range(len(CASES)))
def test_three_level_vcycle_fp64(ras, case):
    dims, parts, ov, ov_c, ratios = CASES[case]
    res, J, A = build(dims, seed=3 + case)
    T = oracle_three_level(A, dims, parts, ov, ov_c, ratios)
    gp, pc = gpu_three_level(ras, res, parts, ov, ov_c, ratios)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(res.grid.n, seed)
        z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), T(r)) < 1e-9, seed


@pytest.mark.parametrize("prec,tol", [(32, 5e-3), (16, 5e-2)])
@pytest.mark.parametrize("case", [1, 3])
def test_three_level_reduced_precision(ras, case, prec, tol):
    """FP32 / BF16-stored factors (FP32 solves) and the FP32 coarsest block LU
    against the oracle with factors rounded the same way."""
    dims, parts, ov, ov_c, ratios = CASES[case]
    res, J, A = build(dims, seed=9)
    T = oracle_three_level(A, dims, parts, ov, ov_c, ratios, prec=prec)
    gp, pc = gpu_three_level(ras, res, parts, ov, ov_c, ratios, prec=prec, cprec=32)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 4)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < tol


def test_three_level_is_linear_and_repeatable(ras):
    dims, parts, ov, ov_c, ratios = CASES[1]
    res, J, A = build(dims, seed=21)
    gp, pc = gpu_three_level(ras, res, parts, ov, ov_c, ratios)
    pc.factor(j_to_dev(J))
    n = res.grid.n
    r1, r2 = syn.random_vector(n, 1), syn.random_vector(n, 2)
    outs = []
    for r in (r1, r2, 2.0 * r1 - 3.0 * r2, r1):
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        outs.append(host(z))
    assert rel_err(outs[2], 2.0 * outs[0] - 3.0 * outs[1]) < 1e-12
    assert np.array_equal(outs[0], outs[3])          # deterministic


def test_three_level_newton_step_matches_oracle(ras):
    res = syn.small_3d(24, 20, 16, seed=11)
    g = res.grid
    dims, parts, ov, ov_c, ratios = (g.nx, g.ny, g.nz), (3, 2, 2), 1, 1, (2, 2, 2)
    prob = disc.Problem(res)

    def fac(A, J):
        return oracle_three_level(A, dims, parts, ov, ov_c, ratios)

    p0 = np.full(g.n, res.p0)
    x_ref, info = newton.newton_solve(prob, fac, p0, p0, res.dt, 1)
    gp, pc = gpu_three_level(ras, res, parts, ov, ov_c, ratios)
    p = dev(p0)
    out = gp.newton_step(pc, p, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    assert out["newton_iters"] == info["newton_iters"]
    assert out["lin_iters"] == info["lin_iters"]
    fh = np.array(out["fnorm_history"])
    ref = np.array(info["fnorm_history"])
    assert np.all(np.abs(fh - ref) <= 1e-9 * ref + 1e-12 * ref[0])
    assert rel_err(host(p), x_ref) < 1e-10


def test_three_level_fewer_iterations_than_one_level(ras):
    res = syn.small_3d(48, 48, 16, seed=13)
    g = res.grid
    gp = ras.Problem(res)
    p = dev(syn.random_pressure(res, 2, 1.0, 3.0))
    p0 = dev(np.full(g.n, res.p0))
    F = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p0, p0, res.dt, 1, F, gp.J)
    its = {}
    for nl in (1, 3):
        pc = ras.Precond(gp, (4, 4, 2), 1, factor_prec=32, nlevels=nl, coarsen=(2, 2, 2),
                         coarse_prec=32, coarse_overlap=1)
        pc.factor(gp.J)
        x = torch.zeros_like(F)
        its[nl] = gp.gmres_solve(gp.J, pc, -F, x, rtol=1e-6, maxit=2000)["iters"]
    assert its[3] < its[1]


def test_three_level_rejects_other_combinations(ras):
    res = syn.small_3d(16, 16, 8, seed=2)
    gp = ras.Problem(res)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, nlevels=3, coarsen=(2, 2, 2), mlevel_type=1)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, nlevels=4, coarsen=(2, 2, 2))
