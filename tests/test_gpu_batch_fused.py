"""The batched solver (ras_batch_*: every FGMRES operation of all reservoirs in
one launch) against the single-reservoir routines and the oracle: the same
FGMRES iterates for a fixed number of iterations, per-reservoir convergence,
implicit steps that meet the oracle's Newton test and agree with newton_step,
and the handle checks."""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev, rel_err

pytestmark = pytest.mark.gpu

DIMS = [(12, 10, 8), (16, 14, 6), (9, 11, 7)]


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def reservoirs():
    return [syn.small_3d(*d, seed=20 + i) for i, d in enumerate(DIMS)]


def make_pc(ras, gp, prec, nlevels, parts=(2, 2, 2)):
    if nlevels == 1:
        return ras.Precond(gp, parts, 1, factor_prec=prec)
    return ras.Precond(gp, parts, 1, factor_prec=prec, nlevels=2, coarsen=(2, 2, 2), coarse_prec=prec)


def setup(ras, prec=64, nlevels=1):
    out = []
    for r in reservoirs():
        prob = disc.Problem(r)
        p = syn.random_pressure(r, 3)
        _, J = disc.residual(prob, p, 0.99 * p, 0.98 * p, r.dt, 2, want_jac=True)
        gp = ras.Problem(r)
        pc = make_pc(ras, gp, prec, nlevels)
        Jd = j_to_dev(J)
        pc.factor(Jd)
        b = dev(syn.random_vector(r.grid.n, 5))
        out.append((r, prob, J, gp, pc, Jd, b))
    return out


@pytest.mark.parametrize("prec,nlevels", [(64, 1), (32, 1), (64, 2), (32, 2)])
def test_fixed_iterations_match_single(ras, prec, nlevels):
    """12 iterations (restart 10, tolerance unreachable): the same iterates as
    gmres_solve up to the order of the reductions' sums (one level, and the
    two-level V-cycle with the exact coarse solve)."""
    items = setup(ras, prec, nlevels)
    bs = ras.BatchSolver([it[3] for it in items], [it[4] for it in items])
    xs = [torch.zeros_like(it[6]) for it in items]
    outs = bs.gmres([it[5] for it in items], [it[6] for it in items], xs, restart=10, maxit=12, rtol=1e-300)
    for it, x, o in zip(items, xs, outs):
        gp, pc, Jd, b = it[3], it[4], it[5], it[6]
        x1 = torch.zeros_like(b)
        o1 = gp.gmres_solve(Jd, pc, b, x1, restart=10, maxit=12, rtol=1e-300)
        assert o["iters"] == o1["iters"] == 12
        assert rel_err(host(x), host(x1)) < 1e-10
        assert rel_err(np.array(o["history"]), np.array(o1["history"])) < 1e-9


def test_each_reservoir_converges_on_its_own(ras):
    items = setup(ras, 32)
    bs = ras.BatchSolver([it[3] for it in items], [it[4] for it in items])
    xs = [torch.zeros_like(it[6]) for it in items]
    outs = bs.gmres([it[5] for it in items], [it[6] for it in items], xs, restart=30, maxit=500, rtol=1e-9)
    iters = []
    for it, x, o in zip(items, xs, outs):
        r, J, b = it[0], it[2], it[6]
        A = disc.jacobian_csr(r.grid, J)
        res = np.linalg.norm(host(b) - A @ host(x))
        assert o["converged"]
        assert res <= 1e-9 * np.linalg.norm(host(b)) * 1.01
        x1 = torch.zeros_like(b)
        o1 = it[3].gmres_solve(it[5], it[4], b, x1, restart=30, maxit=500, rtol=1e-9)
        assert abs(o["iters"] - o1["iters"]) <= 1
        iters.append(o["iters"])
    assert len(set(iters)) > 1            # the reservoirs stopped at different iterations


@pytest.mark.parametrize("nlevels", [1, 2])
def test_newton_steps_match_single_and_oracle(ras, nlevels):
    """Two implicit steps (BDF1 then BDF2) of three reservoirs batched vs
    newton_step per reservoir; every batched state meets the oracle's Newton test."""
    res = reservoirs()
    probs = [ras.Problem(r) for r in res]
    pcs = [make_pc(ras, gp, 32, nlevels) for gp in probs]
    bs = ras.BatchSolver(probs, pcs)
    p0 = [torch.full((r.grid.n,), r.p0, dtype=torch.float64, device="cuda") for r in res]
    pl, plm1 = [p.clone() for p in p0], [p.clone() for p in p0]
    ql, qlm1 = [p.clone() for p in p0], [p.clone() for p in p0]
    for step in range(2):
        order = 1 if step == 0 else 2
        ps = [p.clone() for p in pl]
        st, outs = bs.newton_step(ps, pl, plm1 if order == 2 else None, [r.dt for r in res], order)
        assert st == 0
        for i, r in enumerate(res):
            q = ql[i].clone()
            o1 = probs[i].newton_step(pcs[i], q, ql[i], qlm1[i], r.dt, order)
            assert o1["status"] == 0
            assert rel_err(host(ps[i]), host(q)) < 1e-7
            prob = disc.Problem(r)
            a, b_, c = host(ps[i]), host(pl[i]), host(plm1[i])
            f0 = np.linalg.norm(disc.residual(prob, b_, b_, c, r.dt, order))
            f1 = np.linalg.norm(disc.residual(prob, a, b_, c, r.dt, order))
            assert f1 <= max(1e-6 * f0, 1e-10) * 1.01
            assert outs[i]["newton_iters"] >= 1
            qlm1[i], ql[i] = ql[i], q
        plm1, pl = pl, ps


def _two_steps(ras, env):
    """Two batched implicit steps (BDF1, BDF2) of the three reservoirs, two-level FP32,
    with the batch handle created under env."""
    import os
    res = reservoirs()
    probs = [ras.Problem(r) for r in res]
    pcs = [make_pc(ras, gp, 32, 2) for gp in probs]
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        bs = ras.BatchSolver(probs, pcs)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
    pl = [torch.full((r.grid.n,), r.p0, dtype=torch.float64, device="cuda") for r in res]
    plm1 = [p.clone() for p in pl]
    for step in range(2):
        order = 1 if step == 0 else 2
        ps = [p.clone() for p in pl]
        st, _ = bs.newton_step(ps, pl, plm1 if order == 2 else None, [r.dt for r in res], order)
        assert st == 0
        plm1, pl = pl, ps
    return pl


def test_elimination_waves_do_not_change_bits(ras):
    """The batched block eliminations give the same states whether the reservoirs share
    one cooperative launch (the default for three reservoirs) or each takes a launch of
    its own with every CTA (RAS_COARSE_WAVE_CTAS larger than the grid)."""
    a = _two_steps(ras, {})
    b = _two_steps(ras, {"RAS_COARSE_WAVE_CTAS": "100000"})
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_batch_handle_checks(ras):
    res = reservoirs()[:2]
    probs = [ras.Problem(r) for r in res]
    one = [ras.Precond(gp, (2, 2, 2), 1, factor_prec=32) for gp in probs]
    two = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32)
    kas = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_prec=32,
                      mlevel_type=1)
    itc = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=32, nlevels=2, coarsen=(2, 2, 2), coarse_solver=1)
    three = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=32, nlevels=3, coarsen=(2, 2, 2), coarse_prec=32)
    asm = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=32, ras_type=0)
    f64 = ras.Precond(probs[1], (2, 2, 2), 1, factor_prec=64)
    for pcs in ([one[0], two], [one[0], kas], [one[0], itc], [one[0], three], [one[0], asm], [one[0], f64],
                [one[0], one[0]]):
        with pytest.raises(ras.RasError):
            ras.BatchSolver(probs, pcs)
    with pytest.raises(ras.RasError):
        ras.BatchSolver([probs[0], probs[0]], [one[0], one[0]])


def test_batch_module_fused_equals_streams(ras):
    """The batch module's fused driver and its one-stream-per-reservoir driver
    reach the same states (to the solvers' tolerances) for uneven sizes."""
    from paper_2007_13966_gb300 import batch

    def make(n, i):
        return syn.lognormal_reservoir(n, n, n, 0.8 * n, 0.8 * n, 0.8 * n, sigma=1.0, corr=4.0,
                                       seed_k=300 + i, seed_phi=400 + i)

    res = batch.random_batch(5, 10, 22, 11, make)
    fused = batch.solve_batch(res, 2, batch.BatchOpts(box=8, fused=True))
    streams = batch.solve_batch(res, 2, batch.BatchOpts(box=8, threads=4, fused=False))
    for (pf, itf), (ps, its) in zip(fused, streams):
        assert rel_err(host(pf), host(ps)) < 1e-7
        assert [a for a, _ in itf] == [a for a, _ in its]    # Newton iterations per step


@pytest.mark.parametrize("prec,nlevels", [(32, 1), (32, 2)])
def test_graph_cycle_equals_direct_launches(ras, prec, nlevels):
    """A restart cycle of the batched FGMRES (every reservoir's Arnoldi scalars on the
    device, no host round trip) replayed as a CUDA graph gives the same bits as the
    same launches issued one by one (RAS_BATCH_GRAPH=0), over several restarts and
    with reservoirs stopping at different iterations."""
    import os
    items = setup(ras, prec, nlevels)
    outs, xs_all = [], []
    for graph in ("1", "0"):
        old = os.environ.get("RAS_BATCH_GRAPH")
        os.environ["RAS_BATCH_GRAPH"] = graph
        try:
            bs = ras.BatchSolver([it[3] for it in items], [it[4] for it in items])
            xs = [torch.zeros_like(it[6]) for it in items]
            outs.append(bs.gmres([it[5] for it in items], [it[6] for it in items], xs, restart=8,
                                 maxit=200, rtol=1e-9))
            xs_all.append(xs)
            del bs
        finally:
            if old is None:
                del os.environ["RAS_BATCH_GRAPH"]
            else:
                os.environ["RAS_BATCH_GRAPH"] = old
    for a, b in zip(outs[0], outs[1]):
        assert a["iters"] == b["iters"] and a["history"] == b["history"]
    for xa, xb in zip(*xs_all):
        assert torch.equal(xa, xb)
    if nlevels == 1:   # one level: the reservoirs stop at different iterations (device masks)
        assert len({o["iters"] for o in outs[0]}) > 1
