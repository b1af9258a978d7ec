"""The subdomain solves' level schedule is a performance setting only (every
schedule gives bit-identical results), invalid schedules are refused without
changing the handle, and the measuring autotuners return a candidate of their
table that solves the problem."""
import pytest
import torch

from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def factored(ras, prec=32, nlevels=1):
    r = syn.small_3d(24, 20, 12, seed=4)
    N = r.grid.n
    gp = ras.Problem(r)
    pc = ras.Precond(gp, (2, 2, 1), 2, factor_prec=prec, nlevels=nlevels, coarsen=(2, 2, 2), coarse_prec=prec)
    p = dev(syn.random_pressure(r, 3))
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    gp.residual_eval(p, p, p, r.dt, 1, F, gp.J)
    pc.factor(gp.J)
    return r, gp, pc, dev(syn.random_vector(N, 6))


@pytest.mark.parametrize("prec,nlevels", [(32, 1), (64, 1), (16, 1), (32, 2)])
def test_schedules_give_identical_results(ras, prec, nlevels):
    r, gp, pc, v = factored(ras, prec, nlevels)
    z0 = torch.zeros_like(v)
    pc.apply(v, z0)
    default = pc.schedule()
    for chunk, threads in [(256, 0), (512, 128), (2048, 64), (0, 256)]:
        try:
            pc.set_schedule(chunk, threads)
        except ras.RasError:
            continue
        z = torch.zeros_like(v)
        pc.apply(v, z)
        assert torch.equal(z, z0), (chunk, threads)
    pc.set_schedule(0, 0)
    assert pc.schedule() == default


def test_invalid_schedule_is_refused(ras):
    r, gp, pc, v = factored(ras)
    before = pc.schedule()
    for chunk, threads in [(0, 48), (0, 1024), (-1, 0), (1 << 20, 0)]:
        with pytest.raises(ras.RasError):
            pc.set_schedule(chunk, threads)
        assert pc.schedule() == before


def test_tune_schedule(ras):
    from paper_2007_13966_gb300 import autotune
    r, gp, pc, v = factored(ras)
    z0 = torch.zeros_like(v)
    pc.apply(v, z0)
    best, table = autotune.tune_schedule(pc, v, torch.zeros_like(v), reps=5)
    assert best in [d["schedule"] for d in table]
    assert pc.schedule() == best
    assert min(d["sec"] for d in table) == [d["sec"] for d in table if d["schedule"] == best][0]
    z = torch.zeros_like(v)
    pc.apply(v, z)
    assert torch.equal(z, z0)


def test_tune_box_and_batch(ras):
    from paper_2007_13966_gb300 import autotune, batch
    r = syn.small_3d(24, 20, 12, seed=4)
    box, table = autotune.tune_box(r, boxes=(6, 8, 12))
    assert box in (6, 8, 12) and all(d["converged"] for d in table)

    def make(n, i):
        return syn.lognormal_reservoir(n, n, n, 0.8 * n, 0.8 * n, 0.8 * n, sigma=1.0, corr=4.0,
                                       seed_k=500 + i, seed_phi=600 + i)

    res = batch.random_batch(3, 10, 18, 5, make)
    b = batch.Batch(res, batch.BatchOpts(box=8, fused=True, tune=True))
    assert b.schedule in [d["chunk_cells"] for d in b.tune_table]
    ref = batch.solve_batch(res, 1, batch.BatchOpts(box=8, fused=True))
    b.advance(1)
    for i, (p, _) in zip(b.inst, ref):
        assert torch.equal(i.p_l, p)                 # the schedule does not change the results
