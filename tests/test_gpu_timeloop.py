"""The time loop's step cut (paper_2007_13966_gb300/timeloop.py) around the
library's newton_step on the GPU, with a failure made on the host (a fake step
that rejects one chosen attempt; no GPU fault is involved): the rejected step is
retried at half the size with BDF1, the size grows back, the run lands on t_end,
and every accepted state equals the oracle's implicit step for the same sizes
and orders (FP64 one-level RAS, 1e-10)."""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn
from paper_2007_13966_gb300 import timeloop

from gpu_util import host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def test_step_cut_on_a_host_made_failure(ras):
    res = syn.small_3d(8, 6, 4, seed=3)
    prob = disc.Problem(res)
    g = res.grid
    parts, ov = (2, 2, 1), 1
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=64)
    lib_step = timeloop.newton_stepper(gp, pc)
    calls = []

    def step(p_l, p_lm1, dt, order):
        calls.append((dt, order))
        if len(calls) == 2:                  # the second attempt fails (host-made)
            return None, {"status": 3}
        return lib_step(p_l, p_lm1, dt, order)

    p0 = torch.full((g.n,), res.p0, dtype=torch.float64, device="cuda")

    def copy(t):
        return t.clone()
    p, rec = timeloop.run(step, p0, timeloop.TimeLoopOpts(dt=res.dt, t_end=3 * res.dt, grow_after=2),
                          copy=copy)
    assert rec.cuts == 1
    assert calls[1] == (res.dt, 2) and calls[2] == (0.5 * res.dt, 1)
    assert abs(rec.t[-1] - 3 * res.dt) <= 1e-12 * res.dt
    assert rec.order[0] == 1 and rec.order[1] == 1     # the first step and the restart after the cut
    assert all(info["status"] == 0 for info in rec.info)
    # the oracle's steps with the accepted sizes and orders
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov)
    q_l = np.full(g.n, res.p0)
    q_lm1 = q_l.copy()
    for dt, order in zip(rec.dt, rec.order):
        q, info = newton.newton_solve(prob, fac, q_l, q_lm1 if order == 2 else q_l, dt, order)
        assert info["status"] == 0
        q_lm1, q_l = q_l, q
    assert rel_err(host(p), q_l) < 1e-10
