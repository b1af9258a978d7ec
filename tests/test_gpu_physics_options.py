"""GPU parity of the physics options beyond Eq. gover_sys's base form, against
the oracle (itself pinned in test_oracle_rates.py / test_oracle_conservative.py):
fixed injection rates (the paper's Case-2 fixed injection velocity, Section 4)
and the conservative accumulation form V phi D_t(p/Z). Residual and Jacobian at
1e-12, implicit steps against the oracle's, discrete mass conservation of a
closed domain on the GPU, and the adjoint gradient in the conservative form."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import discretization as disc
from oracle import eos, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, rel_err, STENCIL

pytestmark = pytest.mark.gpu

EMPTY = syn.Connections(np.array([], dtype=np.int32), np.array([]), np.array([]))


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def with_rates(res, seed=3):
    """Rates into the x = 0 face cells of the first z layer (m^3/s, a Darcy
    velocity of 1e-5 m/s through each cell's face)."""
    g = res.grid
    Q = np.zeros(g.n)
    rng = np.random.default_rng(seed)
    for j in range(g.ny):
        Q[g.nx * j] = 1e-5 * g.hy * g.hz * (0.5 + rng.random())
    return dataclasses.replace(res, rate_Q=Q)


VARIANTS = {
    "rates": lambda r: with_rates(r),
    "conservative": lambda r: dataclasses.replace(r, conservative=True),
    "both": lambda r: dataclasses.replace(with_rates(r), conservative=True),
    "conservative-upwind-gravity": lambda r: dataclasses.replace(r, conservative=True, upwind=True,
                                                                  gravity=9.80665),
}


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_residual_and_jacobian(ras, variant, order):
    res = VARIANTS[variant](syn.small_3d(24, 20, 12, seed=11))
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    p = syn.random_pressure(res, 5)
    rng = np.random.default_rng(5)
    p_l = p * (1 - 0.02 * rng.random(p.size))
    p_lm1 = p_l * (1 - 0.02 * rng.random(p.size))
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, order, want_jac=True)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, Fd, gp.J, want_norm=True)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s


@pytest.mark.parametrize("variant", ["rates", "conservative"])
def test_time_steps_match_the_oracle(ras, variant):
    """Three BDF steps (BDF1 then BDF2) with FP64 one-level RAS: Newton and FGMRES
    iteration counts equal, states at 1e-10."""
    res = VARIANTS[variant](syn.small_3d(16, 12, 8, seed=4))
    g = res.grid
    parts, ov = (2, 2, 2), 1
    prob = disc.Problem(res)
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov)
    states, infos = newton.simulate(prob, fac, 3)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=64)
    p_l = dev(states[0])
    p_lm1 = p_l.clone()
    for step in range(3):
        p = p_l.clone()
        out = gp.newton_step(pc, p, p_l, p_lm1, res.dt, 1 if step == 0 else 2)
        assert out["status"] == 0
        assert out["newton_iters"] == infos[step]["newton_iters"]
        assert out["lin_iters"] == infos[step]["lin_iters"]
        assert rel_err(host(p), states[step + 1]) < 1e-10
        p_lm1, p_l = p_l, p


def test_conservative_form_keeps_the_mass_of_a_closed_domain(ras):
    """No connections, no rates: a converged conservative step keeps sum V phi p/Z
    (computed here from the oracle's Z) to the Newton tolerance; the form of
    Eq. gover_sys drifts at O(dt)."""
    base = dataclasses.replace(syn.small_3d(16, 12, 8, seed=3), conns=EMPTY)
    n = base.grid.n
    p0 = 3e6 + 3e6 * np.random.default_rng(2).random(n)
    drift = {}
    for cons in (False, True):
        res = dataclasses.replace(base, conservative=cons)
        prob = disc.Problem(res)
        gp = ras.Problem(res)
        pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32)
        p = dev(p0)
        out = gp.newton_step(pc, p, dev(p0), dev(p0), 10 * res.dt, 1, rtol=1e-12, atol=0.0,
                             lin_rtol=1e-12, lin_atol=0.0)
        fh = out["fnorm_history"]
        assert out["status"] == 0 or fh[-1] <= 1e-10 * fh[0]

        def mass(q):
            Z = eos.eos_state(q, prob.fluid, prob.a, prob.b)[0]
            return np.sum(prob.V * prob.phi * q / Z)
        drift[cons] = abs(mass(host(p)) - mass(p0)) / mass(p0)
    assert drift[True] < 1e-11, drift
    assert drift[False] > 1e-4, drift


def test_conservative_adjoint_gradient_matches_the_oracle(ras):
    from paper_2007_13966_gb300 import adjoint as gadj
    res = dataclasses.replace(syn.small_3d(12, 10, 4, seed=7), conservative=True)
    cells = oadj.producer_cells(res)
    phi_ref, grad_ref, _ = oadj.adjoint_gradient(res, 3, cells)
    theta = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = gadj.objective(theta, res, 3)
    phi.backward()
    assert abs(float(phi.detach()) - phi_ref) <= 1e-10 * phi_ref
    assert rel_err(host(theta.grad), grad_ref) < 1e-7
