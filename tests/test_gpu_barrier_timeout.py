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


def _batch_items(ras):
    out = []
    for i, d in enumerate([(12, 10, 8), (16, 14, 6), (9, 11, 7)]):
        r = syn.small_3d(*d, seed=40 + i)
        prob = disc.Problem(r)
        p = syn.random_pressure(r, 3)
        _, J = disc.residual(prob, p, 0.99 * p, 0.98 * p, r.dt, 2, want_jac=True)
        gp = ras.Problem(r)
        pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
        Jd = j_to_dev(J)
        pc.factor(Jd)
        out.append((gp, pc, Jd, dev(syn.random_vector(r.grid.n, 5)), r.p0))
    return out


def test_batched_barrier_timeout_is_reported_and_recoverable(ras):
    """The same for the batched cooperative coarse solves (a CTA group and a
    barrier word per reservoir, inside the replayed restart-cycle graph): the
    batched FGMRES reports RAS_ETIMEOUT, and the next call with the normal limit
    gives the iterates of a fresh batch bit for bit."""
    items = _batch_items(ras)
    gps, pcs, Js, bs_, p0s = ([it[k] for it in items] for k in range(5))
    bs = ras.BatchSolver(gps, pcs)
    xs = [torch.zeros_like(b) for b in bs_]
    try:
        os.environ["RAS_BARRIER_POLLS"] = "1"
        with pytest.raises(ras.RasError) as ei:
            bs.gmres(Js, bs_, xs, restart=10, maxit=12, rtol=1e-300)
        assert ei.value.status == RAS_ETIMEOUT
    finally:
        del os.environ["RAS_BARRIER_POLLS"]
    try:
        os.environ["RAS_BARRIER_POLLS"] = "1"      # the batched block eliminations (factor waves)
        ps = [torch.full_like(b, p0) for b, p0 in zip(bs_, p0s)]
        with pytest.raises(ras.RasError) as ei:
            bs.newton_step(ps, [p.clone() for p in ps], None, [0.1] * len(ps), 1)
        assert ei.value.status == RAS_ETIMEOUT
    finally:
        del os.environ["RAS_BARRIER_POLLS"]
    torch.cuda.synchronize()
    for pc, J in zip(pcs, Js):                     # the newton step refactored the preconditioners
        pc.factor(J)
    xs = [torch.zeros_like(b) for b in bs_]
    outs = bs.gmres(Js, bs_, xs, restart=10, maxit=12, rtol=1e-300)
    fresh = ras.BatchSolver(gps, pcs)
    xf = [torch.zeros_like(b) for b in bs_]
    outf = fresh.gmres(Js, bs_, xf, restart=10, maxit=12, rtol=1e-300)
    for x, y, o, of in zip(xs, xf, outs, outf):
        assert o["iters"] == of["iters"] == 12
        assert torch.equal(x, y)
        assert np.all(np.isfinite(host(x)))
