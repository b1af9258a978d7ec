"""Many independent reservoirs solved together on one GPU.

Every reservoir has its own problem and preconditioner handles. Two drivers:

* fused (default): one library batch handle (ras_batch_*) advances all
  reservoirs in lock step; every FGMRES operation of all reservoirs (their
  subdomain solves, operators, Arnoldi dot products and updates) is one kernel
  launch, and one host synchronisation per Arnoldi step serves the batch.
* streams: each reservoir on its own CUDA stream, driven by a pool of host
  threads (the library's calls release the interpreter lock; their host
  synchronisations wait on their own stream only).

The Newton / FGMRES scalar logic stays on the host, one Arnoldi step at a time.
"""
from __future__ import annotations

import concurrent.futures as cf
from dataclasses import dataclass

import numpy as np
import torch

from . import ras


@dataclass
class BatchOpts:
    box: int = 16                 # target subdomain edge (cells)
    overlap: int = 1
    factor_prec: int = 32
    threads: int = 8
    rtol: float = 1e-6
    lin_rtol: float = 1e-6
    fused: bool = True            # one batch handle; False: one stream per reservoir
    nlevels: int = 1              # 2: two-level V-cycle with the exact coarse solve
    coarsen: tuple = (4, 4, 4)
    tune: bool = False            # fused: pick the subdomain solves' chunk size by timing


def parts_for(res, box):
    g = res.grid
    return tuple(max(1, min(n, int(round(n / box)))) for n in (g.nx, g.ny, g.nz))


class _Instance:
    def __init__(self, res, opts: BatchOpts, own_stream=True):
        self.res, self.opts = res, opts
        self.stream = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
        with torch.cuda.stream(self.stream):
            self.gp = ras.Problem(res)
            self.pc = ras.Precond(self.gp, parts_for(res, opts.box), opts.overlap,
                                  factor_prec=opts.factor_prec, nlevels=opts.nlevels,
                                  coarsen=opts.coarsen, coarse_prec=opts.factor_prec)
            N = res.grid.n
            self.p_l = torch.full((N,), res.p0, dtype=torch.float64, device="cuda")
            self.p_lm1 = self.p_l.clone()
        self.step = 0
        self.iters = []

    def advance(self, nsteps):
        o = self.opts
        with torch.cuda.stream(self.stream):
            for _ in range(nsteps):
                order = 1 if self.step == 0 else 2
                p = self.p_l.clone()
                out = self.gp.newton_step(self.pc, p, self.p_l, self.p_lm1, self.res.dt, order,
                                          rtol=o.rtol, lin_rtol=o.lin_rtol)
                if out["status"] != 0:
                    raise RuntimeError(f"newton_step status {out['status']}")
                self.iters.append((out["newton_iters"], out["lin_total"]))
                self.p_lm1, self.p_l = self.p_l, p
                self.step += 1
        self.stream.synchronize()


class Batch:
    """Independent reservoirs advanced together, one stream and handle set each."""

    def __init__(self, reservoirs, opts: BatchOpts | None = None):
        self.opts = opts or BatchOpts()
        self.solver = None
        if self.opts.fused:
            self.inst = [_Instance(r, self.opts, own_stream=False) for r in reservoirs]
            self.solver = ras.BatchSolver([i.gp for i in self.inst], [i.pc for i in self.inst])
            self.schedule, self.tune_table = None, None
            if self.opts.tune:
                from .autotune import tune_batch_schedule
                self.schedule, self.tune_table = tune_batch_schedule(self)
        else:
            self.inst = self._map(lambda r: _Instance(r, self.opts), reservoirs)

    def _map(self, fn, items):
        if self.opts.threads <= 1:
            return [fn(x) for x in items]
        with cf.ThreadPoolExecutor(max_workers=self.opts.threads) as ex:
            return list(ex.map(fn, items))

    def advance(self, nsteps):
        if self.solver is None:
            self._map(lambda i: i.advance(nsteps), self.inst)
            return
        o = self.opts
        for _ in range(nsteps):
            step = self.inst[0].step
            order = 1 if step == 0 else 2
            ps = [i.p_l.clone() for i in self.inst]
            st, outs = self.solver.newton_step(
                ps, [i.p_l for i in self.inst], [i.p_lm1 for i in self.inst] if order == 2 else None,
                [i.res.dt for i in self.inst], order, rtol=o.rtol, lin_rtol=o.lin_rtol)
            if st != 0:
                raise RuntimeError(f"ras_batch_newton_step status {st}")
            for i, p, out in zip(self.inst, ps, outs):
                i.iters.append((out["newton_iters"], out["lin_total"]))
                i.p_lm1, i.p_l = i.p_l, p
                i.step += 1

    @property
    def cells(self):
        return sum(i.res.grid.n for i in self.inst)


def solve_batch(reservoirs, nsteps, opts: BatchOpts | None = None):
    """Advance every reservoir nsteps implicit steps; returns [(final state, iters)]."""
    b = Batch(reservoirs, opts)
    b.advance(nsteps)
    return [(i.p_l, i.iters) for i in b.inst]


def random_batch(count, lo, hi, seed, make):
    """count reservoirs with edges drawn uniformly from lo..hi (seeded);
    make(n, i) builds instance i of edge n."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=count)
    return [make(int(n), i) for i, n in enumerate(sizes)]
