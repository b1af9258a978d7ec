"""The FP32 dense coarse block elimination (Section 3.2, the exact coarse solve of
the two-level methods) with the trailing updates of its Gauss-Jordan block
inverses on the tcgen05 tensor cores (three-term TF32 split, FP32 accumulation):
the coarse correction agrees with the CUDA-core form to FP32 rounding and with
the FP64 oracle to the FP32 tolerance, on block sizes with several 128-row tile
pairs and an odd tile count. The same for the cyclic reduction of the block
tridiagonal system (RAS_COARSE_CR=1 at set-up: its dense products on tcgen05),
single and batched. The elimination's bits do not depend on its grid size."""
import os

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


def _with_env(env, make):
    old = {k: os.environ.get(k) for k in env}
    try:
        os.environ.update(env)
        return make()
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _precond(ras, gp, parts, ov, ratios, tc, cr=False, mlevel_type=4):
    env = {"RAS_COARSE_TC": "1" if tc else "0", "RAS_COARSE_CR": "1" if cr else "0"}
    return _with_env(env, lambda: ras.Precond(gp, parts, ov, factor_prec=32, nlevels=2, coarsen=ratios,
                                              mlevel_type=mlevel_type, coarse_prec=32))


# (grid, parts, overlap, ratios): coarse blocks of 2 planes; 12 x 16 and 16 x 32 planes
# give T = 384 (6 tiles: three pairs) and T = 1024 (16 tiles), 20 x 12 planes T = 480 -> 512
@pytest.mark.parametrize("dims,parts,ov,ratios", [
    ((48, 64, 32), (4, 4, 2), 1, (4, 4, 4)),
    ((64, 128, 64), (4, 8, 4), 2, (4, 4, 4)),
    ((40, 24, 24), (2, 2, 2), 1, (2, 2, 2)),
])
def test_tensor_core_inverses_match(ras, dims, parts, ov, ratios):
    nx, ny, nz = dims
    res = syn.small_3d(nx, ny, nz, seed=5)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 5)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    r = dev(syn.random_vector(res.grid.n, 2))
    z = {}
    for tc in (True, False):
        pc = _precond(ras, gp, parts, ov, ratios, tc)
        pc.factor(Jd)
        z[tc] = torch.zeros_like(r)
        pc.apply(r, z[tc])
    assert rel_err(host(z[True]), host(z[False])) < 1e-4
    A = disc.jacobian_csr(res.grid, J)
    P = ml.interpolation(dims, ratios, 2)
    ref = ml.TwoLevel(A, schwarz.Schwarz(A, dims, parts, ov), P, ml.DenseCoarse(ml.galerkin(A, P)),
                      ml.COARSE_ONLY)(host(r))
    assert rel_err(host(z[True]), ref) < 5e-3


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("dims", [(24, 20, 28), (40, 24, 24)])   # 7 blocks of T = 192, 10 of T = 320
def test_factor_grid_size_does_not_change_bits(ras, prec, dims):
    """The block elimination strides its items over the CTAs the cooperative launch
    has: 1, 2 and 3 CTAs (no more than the two chains, so the next pivot tiles are
    inverted by CTAs that also take trailing updates) give the default grid's bits,
    on the tensor path (FP32) and the CUDA-core path (FP64)."""
    nx, ny, nz = dims
    res = syn.small_3d(nx, ny, nz, seed=8)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 8)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    r = dev(syn.random_vector(res.grid.n, 4))
    outs = []
    for ctas in (None, "1", "2", "3"):
        env = {} if ctas is None else {"RAS_COARSE_FACTOR_CTAS": ctas}
        pc = _with_env(env, lambda: ras.Precond(gp, (2, 2, 2), 1, factor_prec=prec, nlevels=2,
                                                coarsen=(2, 2, 2), mlevel_type=4, coarse_prec=prec))
        pc.factor(Jd)
        z = torch.zeros_like(r)
        pc.apply(r, z)
        outs.append(z)
        del pc
    assert torch.isfinite(outs[0]).all()
    for z in outs[1:]:
        assert torch.equal(z, outs[0])


@pytest.mark.parametrize("dims,parts,ov,ratios", [
    ((48, 64, 32), (4, 4, 2), 1, (4, 4, 4)),      # 8 blocks of T = 384
    ((64, 128, 64), (4, 8, 4), 2, (4, 4, 4)),     # 16 blocks of T = 1024
    ((40, 24, 24), (2, 2, 2), 1, (2, 2, 2)),      # 10 blocks of T = 320
    ((24, 20, 28), (2, 2, 2), 1, (2, 2, 2)),      # 7 blocks (an odd count) of T = 192
])
def test_cyclic_reduction_matches(ras, dims, parts, ov, ratios):
    """Cyclic reduction (inverses of the eliminated blocks in concurrent chains,
    the Schur products and new couplings as dense tcgen05 products) against the
    two-ended elimination and the FP64 oracle's dense coarse solve."""
    nx, ny, nz = dims
    res = syn.small_3d(nx, ny, nz, seed=6)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 6)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    r = dev(syn.random_vector(res.grid.n, 3))
    z = {}
    for cr in (True, False):
        pc = _precond(ras, gp, parts, ov, ratios, True, cr)
        pc.factor(Jd)
        z[cr] = torch.zeros_like(r)
        pc.apply(r, z[cr])
    assert rel_err(host(z[True]), host(z[False])) < 1e-4
    A = disc.jacobian_csr(res.grid, J)
    P = ml.interpolation(dims, ratios, 2)
    ref = ml.TwoLevel(A, schwarz.Schwarz(A, dims, parts, ov), P, ml.DenseCoarse(ml.galerkin(A, P)),
                      ml.COARSE_ONLY)(host(r))
    assert rel_err(host(z[True]), ref) < 5e-3


def test_cyclic_reduction_batched(ras):
    """The batched coarse factorisations and solves take the reduction per
    handle (tensor memory held by the batched factor kernel's CTAs): 12 batched
    FGMRES iterations give the single solver's iterates."""
    items = []
    for i, d in enumerate([(24, 20, 28), (20, 24, 16), (16, 16, 24)]):
        r = syn.small_3d(*d, seed=30 + i)
        prob = disc.Problem(r)
        p = syn.random_pressure(r, 3)
        _, J = disc.residual(prob, p, 0.99 * p, 0.98 * p, r.dt, 2, want_jac=True)
        gp = ras.Problem(r)
        pc = _precond(ras, gp, (2, 2, 2), 1, (2, 2, 2), True, True, mlevel_type=0)
        Jd = j_to_dev(J)
        pc.factor(Jd)
        items.append((gp, pc, Jd, dev(syn.random_vector(r.grid.n, 5))))
    bs = ras.BatchSolver([it[0] for it in items], [it[1] for it in items])
    xs = [torch.zeros_like(it[3]) for it in items]
    outs = bs.gmres([it[2] for it in items], [it[3] for it in items], xs, restart=10, maxit=12, rtol=1e-300)
    for (gp, pc, Jd, b), x, o in zip(items, xs, outs):
        x1 = torch.zeros_like(b)
        o1 = gp.gmres_solve(Jd, pc, b, x1, restart=10, maxit=12, rtol=1e-300)
        assert o["iters"] == o1["iters"] == 12
        assert rel_err(host(x), host(x1)) < 1e-10

    # the batched factorisations (waves of the cooperative factor kernel): one
    # implicit step of the batch against newton_step per reservoir
    res = [syn.small_3d(*d, seed=30 + i) for i, d in enumerate([(24, 20, 28), (20, 24, 16), (16, 16, 24)])]
    probs = [ras.Problem(r) for r in res]
    mk = lambda gp: _precond(ras, gp, (2, 2, 2), 1, (2, 2, 2), True, True, mlevel_type=0)
    bs = ras.BatchSolver(probs, [mk(gp) for gp in probs])
    p0 = [torch.full((r.grid.n,), r.p0, dtype=torch.float64, device="cuda") for r in res]
    ps = [p.clone() for p in p0]
    st, _ = bs.newton_step(ps, p0, None, [r.dt for r in res], 1)
    assert st == 0
    for i, r in enumerate(res):
        q = p0[i].clone()
        o1 = probs[i].newton_step(mk(probs[i]), q, p0[i], p0[i], r.dt, 1)
        assert o1["status"] == 0
        assert rel_err(host(ps[i]), host(q)) < 1e-7
