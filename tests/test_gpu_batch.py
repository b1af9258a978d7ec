"""Independent reservoirs solved concurrently (one stream each, a pool of host
threads) give exactly the states of solving them one after another, and each
state meets the oracle's Newton test."""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def make(n, i):
    return syn.lognormal_reservoir(n, n, n, 0.8 * n, 0.8 * n, 0.8 * n, sigma=1.0, corr=4.0,
                                   seed_k=100 + i, seed_phi=200 + i)


def test_concurrent_equals_sequential(ras):
    from paper_2007_13966_gb300 import batch
    res = batch.random_batch(6, 12, 24, 7, make)
    seq = batch.solve_batch(res, 2, batch.BatchOpts(box=8, threads=1, fused=False))
    con = batch.solve_batch(res, 2, batch.BatchOpts(box=8, threads=4, fused=False))
    for (ps, its), (pc, itc) in zip(seq, con):
        assert its == itc
        assert torch.equal(ps, pc)                      # deterministic per instance


def test_batch_states_meet_newton_test(ras):
    from paper_2007_13966_gb300 import batch
    res = batch.random_batch(4, 10, 20, 3, make)
    out = batch.solve_batch(res, 1, batch.BatchOpts(box=8, threads=4, fused=False))
    for r, (p, _) in zip(res, out):
        prob = disc.Problem(r)
        p0 = np.full(r.grid.n, r.p0)
        f0 = np.linalg.norm(disc.residual(prob, p0, p0, p0, r.dt, 1))
        f1 = np.linalg.norm(disc.residual(prob, p.cpu().numpy(), p0, p0, r.dt, 1))
        assert f1 <= max(1e-6 * f0, 1e-10) * 1.01
