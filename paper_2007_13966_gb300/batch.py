"""Many independent reservoirs solved concurrently on one GPU.

Each reservoir has its own problem and preconditioner handles and its own CUDA
stream; a pool of host threads drives the time loops (the library's calls
release the interpreter lock while they run, and their host synchronisations
wait on their own stream only), so the small per-reservoir kernels of
different instances overlap on the device. The Newton / FGMRES scalar logic
stays on the host, one Arnoldi step at a time, so the loops are not captured
into CUDA graphs.
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


def parts_for(res, box):
    g = res.grid
    return tuple(max(1, min(n, int(round(n / box)))) for n in (g.nx, g.ny, g.nz))


class _Instance:
    def __init__(self, res, opts: BatchOpts):
        self.res, self.opts = res, opts
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.gp = ras.Problem(res)
            self.pc = ras.Precond(self.gp, parts_for(res, opts.box), opts.overlap,
                                  factor_prec=opts.factor_prec)
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
        self.inst = self._map(lambda r: _Instance(r, self.opts), reservoirs)

    def _map(self, fn, items):
        if self.opts.threads <= 1:
            return [fn(x) for x in items]
        with cf.ThreadPoolExecutor(max_workers=self.opts.threads) as ex:
            return list(ex.map(fn, items))

    def advance(self, nsteps):
        self._map(lambda i: i.advance(nsteps), self.inst)

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
