"""Measuring autotuner for the Schwarz preconditioner's subdomain solves.

Two kinds of knob, both chosen by timing on the GPU:

* the level schedule of the subdomain solves (wavefront levels staged per
  shared-memory ring slot, threads per box): a performance setting only, the
  preconditioner's values do not change. Timed on ras_apply for one handle, or
  on a fixed number of batched FGMRES iterations for a batch of reservoirs.
* the subdomain (box) edge: it changes the preconditioner and so the iteration
  counts, so it is timed on a whole linear solve (factorisation included) of
  the first Newton system of an implicit step.

Every function returns the best candidate and the whole timing table.
"""
from __future__ import annotations

import torch

from . import ras

CHUNKS = (256, 384, 512, 768, 1024, 1536)


def _time(fn, reps, warmup=2):
    for _ in range(warmup):
        fn()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps * 1e-3


def tune_schedule(pc, r, z, chunks=CHUNKS, threads=(0,), reps=20):
    """Best (chunk_cells, threads) for pc's apply; pc is left on it."""
    table = []
    for c in chunks:
        for t in threads:
            try:
                pc.set_schedule(c, t)
            except ras.RasError:
                continue                       # shared memory over the limit, bad thread count
            table.append({"schedule": pc.schedule(), "sec": _time(lambda: pc.apply(r, z), reps)})
    if not table:
        raise RuntimeError("no valid schedule among the candidates")
    best = min(table, key=lambda d: d["sec"])
    pc.set_schedule(*best["schedule"])
    return best["schedule"], table


def tune_batch_schedule(batch, chunks=CHUNKS, iters=6):
    """Best chunk size for every reservoir of a fused batch (batch.Batch), timed on
    `iters` batched FGMRES iterations on each reservoir's first Newton system; the
    batch is left on it (with a new batch handle)."""
    insts = batch.inst
    Js, bs = [], []
    for i in insts:
        N = i.res.grid.n
        F = torch.zeros(N, dtype=torch.float64, device="cuda")
        i.gp.residual_eval(i.p_l, i.p_l, i.p_lm1, i.res.dt, 1, F, i.gp.J)
        i.pc.factor(i.gp.J)
        Js.append([c.clone() for c in i.gp.J])
        bs.append(-F)
    xs = [torch.zeros_like(b) for b in bs]
    table = []
    for c in chunks:
        try:
            for i in insts:
                i.pc.set_schedule(c, 0)
        except ras.RasError:
            continue
        solver = ras.BatchSolver([i.gp for i in insts], [i.pc for i in insts])
        sec = _time(lambda: solver.gmres(Js, bs, xs, restart=30, maxit=iters, rtol=1e-300), 2, warmup=1)
        table.append({"chunk_cells": c, "sec_per_iter": sec / iters})
        del solver
    if not table:
        raise RuntimeError("no valid schedule among the candidates")
    best = min(table, key=lambda d: d["sec_per_iter"])
    for i in insts:
        i.pc.set_schedule(best["chunk_cells"], 0)
    batch.solver = ras.BatchSolver([i.gp for i in insts], [i.pc for i in insts])
    return best["chunk_cells"], table


def tune_box(res, boxes=(8, 12, 16, 20, 24), overlap=1, factor_prec=32, nlevels=1,
             coarsen=(4, 4, 4), rtol=1e-6):
    """Best box edge for the reservoir `res`: each candidate factors the Jacobian
    of the first Newton system of a BDF1 step from the initial state and solves
    it to rtol with FGMRES(30); the fastest factorisation + solve wins."""
    from .batch import parts_for
    N = res.grid.n
    gp = ras.Problem(res)
    p0 = torch.full((N,), res.p0, dtype=torch.float64, device="cuda")
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    gp.residual_eval(p0, p0, p0, res.dt, 1, F, gp.J)
    b = -F
    table = []
    for box in boxes:
        parts = parts_for(res, box)
        try:
            pc = ras.Precond(gp, parts, overlap, factor_prec=factor_prec, nlevels=nlevels, coarsen=coarsen,
                             coarse_prec=factor_prec)
        except ras.RasError:
            continue
        x = torch.zeros_like(b)
        out = {}

        def run():
            pc.factor(gp.J)
            x.zero_()
            out.update(gp.gmres_solve(gp.J, pc, b, x, restart=30, maxit=2000, rtol=rtol))

        sec = _time(run, 2, warmup=1)
        table.append({"box": box, "parts": parts, "sec": sec, "iters": out["iters"],
                      "converged": out["converged"]})
        del pc
    ok = [d for d in table if d["converged"]]
    if not ok:
        raise RuntimeError("no box size converged")
    best = min(ok, key=lambda d: d["sec"])
    return best["box"], table
