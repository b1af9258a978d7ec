"""The time loop's step-cut policy on the CPU, with the oracle's Newton as the step
and failures made on the host (a fake that rejects chosen attempts): without
failures it is the paper's fixed-step loop (BDF1, then BDF2); a failure halves
the step and restarts with BDF1; the step grows back to the target after
`grow_after` accepted steps; the last step lands on t_end; every accepted state
meets the oracle's Newton test for its step size, order and history."""
import numpy as np
import pytest

from oracle import discretization as disc
from oracle import newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn
from paper_2007_13966_gb300 import timeloop


def problem():
    res = syn.small_3d(8, 6, 4, seed=3)
    return res, disc.Problem(res)


def oracle_step(prob, log, reject=()):
    g = prob.grid
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), (2, 2, 1), 1)

    def step(p_l, p_lm1, dt, order):
        log.append((dt, order))
        if len(log) in reject:                       # the fake failing call
            return None, {"status": 3}
        p, info = newton.newton_solve(prob, fac, p_l, p_lm1 if order == 2 else p_l, dt, order)
        return (p if info["status"] == 0 else None), {"history": (p_l, p_lm1, dt, order)}
    return step


def meets_newton_test(prob, p, p_l, p_lm1, dt, order):
    f0 = np.linalg.norm(disc.residual(prob, p_l, p_l, p_lm1 if order == 2 else p_l, dt, order))
    f1 = np.linalg.norm(disc.residual(prob, p, p_l, p_lm1 if order == 2 else p_l, dt, order))
    return f1 <= max(1e-6 * f0, 1e-10) * 1.01


def test_without_failures_it_is_the_fixed_step_loop():
    res, prob = problem()
    log = []
    p0 = np.full(res.grid.n, res.p0)
    p, rec = timeloop.run(oracle_step(prob, log), p0, timeloop.TimeLoopOpts(dt=res.dt, t_end=4 * res.dt))
    assert rec.order == [1, 2, 2, 2] and rec.cuts == 0
    assert np.allclose(rec.dt, res.dt, rtol=0, atol=0)
    # the same steps by hand
    g = prob.grid
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), (2, 2, 1), 1)
    q_l, q_lm1 = p0, p0
    for k in range(4):
        q, _ = newton.newton_solve(prob, fac, q_l, q_lm1, res.dt, 1 if k == 0 else 2)
        q_lm1, q_l = q_l, q
    assert np.array_equal(p, q_l)


def test_failure_halves_restarts_and_grows_back():
    res, prob = problem()
    log = []
    p0 = np.full(res.grid.n, res.p0)
    opts = timeloop.TimeLoopOpts(dt=res.dt, t_end=5 * res.dt, grow_after=2)
    p, rec = timeloop.run(oracle_step(prob, log, reject={3}), p0, opts)
    dt = res.dt
    # attempts: BDF1 dt, BDF2 dt, BDF2 dt rejected, BDF1 dt/2, BDF2 dt/2 (two accepted at
    # the reduced size), BDF1 dt (grown back), BDF2 dt, reaching t = 5 dt
    assert log == [(dt, 1), (dt, 2), (dt, 2), (dt / 2, 1), (dt / 2, 2), (dt, 1), (dt, 2)]
    assert rec.cuts == 1 and rec.order == [1, 2, 1, 2, 1, 2]
    assert abs(rec.t[-1] - opts.t_end) <= 1e-12 * opts.t_end
    # each accepted step started from the previous accepted state
    nxt = [i["history"][0] for i in rec.info[1:]] + [p]
    prev = p0
    for info, p_new in zip(rec.info, nxt):
        assert np.array_equal(info["history"][0], prev)
        prev = p_new


def test_every_accepted_state_meets_its_newton_test():
    res, prob = problem()
    log = []
    p0 = np.full(res.grid.n, res.p0)
    opts = timeloop.TimeLoopOpts(dt=res.dt, t_end=3.3 * res.dt, grow_after=1)
    p, rec = timeloop.run(oracle_step(prob, log, reject={2, 3}), p0, opts)
    assert rec.cuts == 2
    assert rec.dt[-1] < res.dt and rec.order[-1] == 1          # shortened last step
    assert abs(sum(rec.dt) - opts.t_end) <= 1e-12 * opts.t_end
    nxt = [i["history"][0] for i in rec.info[1:]] + [p]
    for info, p_new in zip(rec.info, nxt):
        p_l, p_lm1, h, order = info["history"]
        assert meets_newton_test(prob, p_new, p_l, p_lm1, h, order)


def test_cut_below_the_minimum_raises():
    res, prob = problem()
    p0 = np.full(res.grid.n, res.p0)
    step = lambda p_l, p_lm1, dt, order: (None, {})
    with pytest.raises(RuntimeError):
        timeloop.run(step, p0, timeloop.TimeLoopOpts(dt=res.dt, t_end=res.dt, dt_min=res.dt / 8))


class _Tensor(np.ndarray):
    def clone(self):
        return self.copy()


class FakeProblem:
    """Stands in for the library's problem handle: newton_step writes the new state
    into p and returns a status (3, a line-search failure, for chosen calls)."""

    def __init__(self, fail_calls):
        self.calls, self.fail_calls, self.seen = 0, fail_calls, []

    def newton_step(self, pc, p, p_l, p_lm1, dt, order, **kw):
        self.calls += 1
        self.seen.append((p_lm1 is None, order, kw))
        assert p is not p_l and np.array_equal(p, p_l)       # initial guess: a copy of p^l
        p += dt                                               # any state change
        return {"status": 3 if self.calls in self.fail_calls else 0}


def test_newton_stepper_glue():
    gp = FakeProblem({2})
    step = timeloop.newton_stepper(gp, pc=None, rtol=1e-8)
    p0 = np.zeros(3).view(_Tensor)
    p, rec = timeloop.run(step, p0, timeloop.TimeLoopOpts(dt=1.0, t_end=3.0, grow_after=1),
                          copy=lambda t: t.clone())
    # dt 1 (BDF1), dt 1 (BDF2) rejected, dt 1/2 (BDF1), grown: dt 1 (BDF1), last 1/2 (BDF1)
    assert rec.cuts == 1 and rec.order == [1, 1, 1, 1] and rec.dt == [1.0, 0.5, 1.0, 0.5]
    assert np.allclose(p, 3.0)                                 # the accepted increments sum to t_end
    assert all(kw == {"rtol": 1e-8} for _, _, kw in gp.seen)
    assert all(none == (order == 1) for none, order, _ in gp.seen)   # BDF1 gets no p^{l-1}
