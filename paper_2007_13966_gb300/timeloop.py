"""Implicit time loop with a time-step cut on Newton failure.

The paper advances with a fixed step: BDF1 for the first step, then BDF2
(Eqs. implicit-method-bdf1 / -bdf2). Its fixed-step BDF2 formula assumes the two
previous states are one step apart, so after any change of the step size this
loop takes one BDF1 step at the new size before returning to BDF2. Policy:

* a failed step (Newton did not meet its test) is retried from the same state
  with half the step size (BDF1), down to dt_min (then the loop raises);
* after `grow_after` accepted steps at a reduced size the step is doubled again
  (capped by the target dt), again restarting with BDF1;
* the last step is shortened to land on t_end.

The step function is the caller's: step(p_l, p_lm1, dt, order) -> (p or None,
info), None meaning failure; `newton_stepper` builds one from the library's
newton_step.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class TimeLoopOpts:
    dt: float                     # target step size (the paper's fixed dt)
    t_end: float
    dt_min: float | None = None   # default dt / 1024
    grow_after: int = 3           # accepted steps at a reduced size before doubling


@dataclass
class TimeLoopRecord:
    t: list = field(default_factory=list)       # time after each accepted step
    dt: list = field(default_factory=list)
    order: list = field(default_factory=list)
    cuts: int = 0
    info: list = field(default_factory=list)


def run(step, p0, opts: TimeLoopOpts, copy=lambda p: p.copy()):
    """Advance p0 from t = 0 to opts.t_end; returns (final state, record)."""
    dt_min = opts.dt_min if opts.dt_min is not None else opts.dt / 1024
    rec = TimeLoopRecord()
    t, dt = 0.0, opts.dt
    p_l, p_lm1 = copy(p0), None
    restart = True                # the next step is BDF1 (no history at this step size)
    at_size = 0                   # accepted steps at the current reduced size
    eps = 1e-12 * opts.t_end
    while t < opts.t_end - eps:
        h = min(dt, opts.t_end - t)
        last = h < dt             # a shortened final step is a change of size
        order = 1 if (restart or last or p_lm1 is None) else 2
        p, info = step(p_l, p_lm1, h, order)
        if p is None:
            rec.cuts += 1
            dt *= 0.5
            if dt < dt_min:
                raise RuntimeError(f"time step cut below dt_min at t = {t}")
            restart, at_size = True, 0
            continue
        rec.t.append(t + h)
        rec.dt.append(h)
        rec.order.append(order)
        rec.info.append(info)
        t += h
        p_lm1, p_l = p_l, p
        restart = False
        if dt < opts.dt:
            at_size += 1
            if at_size >= opts.grow_after:
                dt = min(2.0 * dt, opts.dt)
                restart, at_size = True, 0
    return p_l, rec


def newton_stepper(gp, pc, **newton_opts):
    """A step function on the library's newton_step (problem gp, preconditioner pc);
    a step fails unless the Newton test was met."""
    def step(p_l, p_lm1, dt, order):
        p = p_l.clone()
        out = gp.newton_step(pc, p, p_l, p_lm1 if order == 2 else None, dt, order, **newton_opts)
        return (p if out["status"] == 0 else None), out
    return step
