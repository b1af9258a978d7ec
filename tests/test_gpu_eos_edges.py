"""GPU Peng-Robinson evaluation at the edges of the method (Section 2, Eq. equ:PR):
a subcritical fluid whose cubic has three real roots over a pressure range
(the largest, vapour root is the admissible one), and states without an
admissible root, reported as RAS_ENOROOT."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import eos
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, rel_err, STENCIL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def subcritical_reservoir(T=150.0):
    res = syn.small_3d(24, 20, 12, seed=11)
    return dataclasses.replace(res, fluid=syn.Fluid(T=T))


def three_root_range(fluid):
    """Pressures (Pa) at which the cubic has three real roots, found here with
    companion-matrix eigenvalues (independent of the oracle's closed form)."""
    a, b = eos.pr_constants(fluid)
    ps = np.geomspace(1e4, 3e7, 3000)
    three = []
    for p in ps:
        A, B = eos.AB(p, a, b, fluid.R, fluid.T)
        r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        if np.all(np.abs(r.imag) < 1e-12):
            three.append(p)
    return min(three), max(three)


@pytest.mark.parametrize("order", [1, 2])
def test_subcritical_residual_and_jacobian_match_the_oracle(ras, order):
    """T = 150 K < T_c: most cells lie where the cubic has three real roots
    (vapour root taken), the rest above the range (one root); residual and
    Jacobian against the oracle at 1e-12 of the array's maximum."""
    res = subcritical_reservoir()
    lo, hi = three_root_range(res.fluid)
    assert lo < 2e5 and 1.5e6 < hi < 2.5e6
    rng = np.random.default_rng(3)
    n = res.grid.n
    # 80 %: inside the three-root range (kept 5 % off its upper end, where the
    # vapour and middle roots merge and dZ/dp is unbounded), 20 %: above it
    p = np.where(rng.random(n) < 0.8, rng.uniform(2e5, 0.95 * hi, n), rng.uniform(1.05 * hi, 4e6, n))
    p_l = p * (1 - 0.01 * rng.random(n))
    p_lm1 = p_l * (1 - 0.01 * rng.random(n))
    prob = disc.Problem(res)
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, order, want_jac=True)
    assert np.all(np.isfinite(F))
    gp = ras.Problem(res)
    Fd = torch.zeros(n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, Fd, gp.J, want_norm=True)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


def test_three_root_cells_take_the_vapour_root(ras):
    """Single-cell problems (no neighbours, no connections): F = V phi c(p) (p - p_l)/dt
    isolates c(p) = (p/Z)(1/p - Z'/Z) of the chosen root, compared with c of the largest
    companion-matrix root; the liquid root's c differs by orders of magnitude."""
    base = subcritical_reservoir()
    f = base.fluid
    a, b = eos.pr_constants(f)
    lo, hi = three_root_range(f)
    ps = np.geomspace(3e5, 0.97 * hi, 40)
    g = syn.Grid(1, 1, 1, 1.0, 1.0, 1.0)
    one = np.ones(1)
    res = syn.Reservoir(grid=g, fluid=f, kx=one * 1e-13, ky=one * 1e-13, kz=one * 1e-13, phi=one * 0.2,
                        conns=syn.Connections(np.zeros(0, np.int32), np.zeros(0), np.zeros(0)))
    gp = ras.Problem(res)
    Fd = torch.zeros(1, dtype=torch.float64, device="cuda")
    for p in ps:
        A, B = eos.AB(p, a, b, f.R, f.T)
        r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        Zv, Zl = r.real.max(), r.real.min()
        dZv = eos.dz_dp_implicit(Zv, p, a, b, f.R, f.T)
        dZl = eos.dz_dp_implicit(Zl, p, a, b, f.R, f.T)
        cv = (p / Zv) * (1 / p - dZv / Zv)
        cl = (p / Zl) * (1 / p - dZl / Zl)
        assert abs(cl - cv) > 0.5 * abs(cv)
        pl = 0.5 * p
        gp.residual_eval(dev(np.array([p])), dev(np.array([pl])), None, 1.0, 1, Fd)
        c_gpu = host(Fd)[0] / (0.2 * (p - pl))
        assert abs(c_gpu - cv) <= 1e-10 * abs(cv), (p, c_gpu, cv, cl)


def test_state_without_an_admissible_root_is_reported(ras):
    """A poisoned cell (NaN pressure, no finite root) gives RAS_ENOROOT from
    residual_eval with the norm requested and from newton_step; the flag is
    cleared, so the next valid call succeeds and matches the oracle."""
    res = syn.small_3d(12, 10, 6, seed=5)
    gp = ras.Problem(res)
    n = res.grid.n
    p = syn.random_pressure(res, 7)
    bad = p.copy()
    bad[n // 3] = np.nan
    Fd = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ras.RasError) as e:
        gp.residual_eval(dev(bad), dev(p), None, res.dt, 1, Fd, want_norm=True)
    assert e.value.status == ras.RAS_ENOROOT
    assert np.isnan(host(Fd)[n // 3])
    # flag cleared: a valid state evaluates normally
    nrm = gp.residual_eval(dev(p), dev(0.99 * p), None, res.dt, 1, Fd, want_norm=True)
    F = disc.residual(disc.Problem(res), p, 0.99 * p, None, res.dt, 1)
    F = F[0] if isinstance(F, tuple) else F
    assert rel_err(host(Fd), F) < 1e-12 and np.isfinite(nrm)
    pc = ras.Precond(gp, (2, 2, 1), 1, factor_prec=64)
    x = dev(bad)
    with pytest.raises(ras.RasError) as e:
        gp.newton_step(pc, x, dev(p), None, res.dt, 1)
    assert e.value.status == ras.RAS_ENOROOT
    x = dev(p)
    out = gp.newton_step(pc, x, dev(p), None, res.dt, 1)
    assert out["status"] == ras.RAS_OK
