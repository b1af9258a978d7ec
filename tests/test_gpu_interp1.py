"""First-order (nearest coarse centre) interpolation, Eq. equ:inter-frist, in the
two-level V-cycle, the inexact coarse solve and the three-level V-cycle, vs
the oracle with the same interpolation."""
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


@pytest.mark.parametrize("ratios", [(2, 2, 2), (4, 3, 2)])
@pytest.mark.parametrize("solver", [0, 1])
def test_two_level_first_order(ras, ratios, solver):
    dims, parts, ov = (24, 18, 12), (3, 2, 2), 1
    res, J, A = build(dims, seed=4)
    P = ml.interpolation(dims, ratios, 1)
    Ac = ml.galerkin(A, P)
    M = schwarz.Schwarz(A, dims, parts, ov)
    if solver == 0:
        C = ml.DenseCoarse(Ac)
    else:
        dc = ml.coarse_dims(dims, ratios)
        C = ml.IterativeCoarse(Ac, dc, tuple(min(p, d) for p, d in zip(parts, dc)), 1, rtol=0.2)
    T = ml.TwoLevel(A, M, P, C, ml.VCYCLE)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=2, coarsen=ratios, coarse_prec=64, interp_order=1,
                     coarse_solver=solver, coarse_rtol=0.2)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 1)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 1e-8


def test_three_level_first_order(ras):
    dims, parts, ov, ov_c, ratios = (24, 20, 16), (2, 2, 2), 1, 1, (2, 2, 2)
    res, J, A = build(dims, seed=6)
    P1 = ml.interpolation(dims, ratios, 1)
    A1 = ml.galerkin(A, P1)
    d1 = ml.coarse_dims(dims, ratios)
    P0 = ml.interpolation(d1, ratios, 1)
    A0 = ml.galerkin(A1, P0)
    T = ml.MultiLevel([A0, A1, A], [None, schwarz.Schwarz(A1, d1, parts, ov_c),
                                    schwarz.Schwarz(A, dims, parts, ov)],
                      [None, P0, P1], ml.DenseCoarse(A0))
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, nlevels=3, coarsen=ratios, coarse_prec=64, interp_order=1,
                     coarse_overlap=ov_c)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 2)
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < 1e-9


def test_third_order_rejected(ras):
    res = syn.small_3d(16, 16, 8, seed=2)
    gp = ras.Problem(res)
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, nlevels=2, coarsen=(2, 2, 2), interp_order=3)
