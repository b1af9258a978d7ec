"""The pencil-wavefront subdomain solves of left-RAS (Eq. equ:as-left): the
x-pencils of a box advance one cell per step, one warp per group of
anti-diagonals, one CTA barrier per step. They must give the same values as the
level-scheduled kernel bit for bit (same arithmetic in the same order, same
records), for every box shape, both reduced precisions, z = M r and z += M r
(inside the two-level V-cycle), and agree with the oracle's emulated storage
precision."""

import numpy as np
import pytest
import torch

from oracle import discretization as disc
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


def _case(dims, seed=5):
    nx, ny, nz = dims
    if nz == 1:
        res = syn.lognormal_reservoir(nx, ny, 1, 50.0, 50.0, 1.0, sigma=1.0, corr=4.0,
                                      seed_k=seed, seed_phi=seed + 1)
    else:
        res = syn.small_3d(nx, ny, nz, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    return res, J


# (grid, parts, overlap): ragged boxes, boxes 24 wide along x, one-cell slabs,
# 2D, a single box, boxes of 20^3 (the 1M workload's interior shape)
CASES = [
    ((24, 20, 12), (3, 2, 2), 1),
    ((17, 13, 9), (3, 3, 2), 2),
    ((40, 30, 20), (2, 3, 2), 2),
    ((17, 9, 7), (17, 1, 1), 1),
    ((64, 64, 1), (4, 4, 1), 1),
    ((12, 10, 8), (1, 1, 1), 0),
    ((32, 32, 32), (2, 2, 2), 2),
]


@pytest.mark.parametrize("prec", [32, 16])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_pencil_equals_level_scheduled(ras, case, prec):
    dims, parts, ov = CASES[case]
    res, J = _case(dims)
    gp = ras.Problem(res)
    a = ras.Precond(gp, parts, ov, factor_prec=prec)
    b = ras.Precond(gp, parts, ov, factor_prec=prec)
    assert b.apply_kernel() == 0          # the default
    a.set_apply_kernel(1)
    assert a.apply_kernel() == 1
    Jd = j_to_dev(J)
    a.factor(Jd)
    b.factor(Jd)
    for seed in (1, 2):
        r = dev(syn.random_vector(res.grid.n, seed))
        za = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
        zb = torch.full_like(za, np.nan)
        a.apply(r, za)
        b.apply(r, zb)
        assert torch.equal(za, zb), float((za - zb).abs().max())


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (16, 2e-2)])
def test_pencil_matches_oracle_emulation(ras, prec, tol):
    dims, parts, ov = CASES[2]
    res, J = _case(dims, seed=9)
    g = res.grid
    A = disc.jacobian_csr(g, J)
    r = syn.random_vector(g.n, 4)
    emu = schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov, prec=prec)(r)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=prec)
    pc.set_apply_kernel(1)
    pc.factor(j_to_dev(J))
    z = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), emu) < tol


@pytest.mark.parametrize("prec", [32, 16])
def test_pencil_accumulate_in_the_v_cycle(ras, prec):
    """The V-cycle's second fine solve accumulates (z += M t): same bits as the
    level-scheduled kernel."""
    dims, parts, ov = (32, 32, 16), (2, 2, 1), 2
    res, J = _case(dims, seed=3)
    gp = ras.Problem(res)
    pcs = []
    for k in (1, 0):
        pc = ras.Precond(gp, parts, ov, factor_prec=prec, nlevels=2, coarsen=(4, 4, 4),
                         coarse_prec=32)
        pc.set_apply_kernel(k)
        pc.factor(j_to_dev(J))
        pcs.append(pc)
    r = dev(syn.random_vector(res.grid.n, 6))
    z = [torch.zeros(res.grid.n, dtype=torch.float64, device="cuda") for _ in pcs]
    for pc, zz in zip(pcs, z):
        pc.apply(r, zz)
    assert torch.equal(z[0], z[1])


def test_kernel_switch_on_the_same_factors(ras):
    """Both kernels read the same records: switching needs no new factorisation."""
    dims, parts, ov = CASES[0]
    res, J = _case(dims)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=32)
    pc.factor(j_to_dev(J))
    r = dev(syn.random_vector(res.grid.n, 1))
    z = [torch.zeros_like(r) for _ in range(3)]
    pc.apply(r, z[0])
    pc.set_apply_kernel(1)
    pc.apply(r, z[1])
    pc.set_apply_kernel(0)
    pc.apply(r, z[2])
    assert torch.equal(z[0], z[1]) and torch.equal(z[1], z[2])
    # FP64 factors and AS / right-RAS stay on the level-scheduled kernel
    with pytest.raises(ras.RasError):
        ras.Precond(gp, parts, ov, factor_prec=64).set_apply_kernel(1)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, parts, ov, factor_prec=32, ras_type=0).set_apply_kernel(1)
