"""The bounded grid barrier of the cooperative coarse kernels: when its wait
runs out (a poll limit far too short for the CTAs to arrive), the kernels stop
and the host reads RAS_ETIMEOUT instead of hanging; the context stays usable
and the next factorisation with the normal limit gives the usual result. No
GPU fault or hang is involved: the limit only shortens a bounded wait."""
import os

import numpy as np
import pytest
import torch

from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev

pytestmark = pytest.mark.gpu

RAS_ETIMEOUT = -7


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def test_barrier_timeout_is_reported_and_recoverable(ras):
    res = syn.small_3d(32, 32, 16, seed=3)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 3)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    Jd = j_to_dev(J)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 2), 1, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
    r = dev(syn.random_vector(res.grid.n, 1))
    try:
        os.environ["RAS_BARRIER_POLLS"] = "1"
        with pytest.raises(ras.RasError) as ei:
            pc.factor(Jd)
        assert ei.value.status == RAS_ETIMEOUT
    finally:
        del os.environ["RAS_BARRIER_POLLS"]
    torch.cuda.synchronize()                       # the context is still usable
    pc.factor(Jd)
    z1 = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(r, z1)
    fresh = ras.Precond(gp, (2, 2, 2), 1, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
    fresh.factor(Jd)
    z2 = torch.zeros_like(z1)
    fresh.apply(r, z2)
    assert torch.equal(z1, z2)
    assert np.all(np.isfinite(host(z1)))
