"""The FP32 dense coarse block elimination (Section 3.2, the exact coarse solve of
the two-level methods) with the trailing updates of its Gauss-Jordan block
inverses on the tcgen05 tensor cores (three-term TF32 split, FP32 accumulation):
the coarse correction agrees with the CUDA-core form to FP32 rounding and with
the FP64 oracle to the FP32 tolerance, on block sizes with several 128-row tile
pairs and an odd tile count."""
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


def _precond(ras, gp, parts, ov, ratios, tc):
    old = os.environ.get("RAS_COARSE_TC")
    try:
        os.environ["RAS_COARSE_TC"] = "1" if tc else "0"
        return ras.Precond(gp, parts, ov, factor_prec=32, nlevels=2, coarsen=ratios, mlevel_type=4,
                           coarse_prec=32)
    finally:
        if old is None:
            del os.environ["RAS_COARSE_TC"]
        else:
            os.environ["RAS_COARSE_TC"] = old


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
