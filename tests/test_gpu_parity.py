"""GPU (CUDA library through the C ABI) vs the CPU FP64 oracle, element by element.

Tolerances: FP64 kernels 1e-12 relative to the array's max; FGMRES/Newton
residual histories 1e-9 relative; states 1e-10 (FP64). Reduced-precision
preconditioners are compared with the oracle's emulation of the same storage
precision (FP32: 1e-5, BF16: 2e-2) and, at the solver level, by the converged
state against the FP64 oracle (1e-6).
"""
import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import krylov, newton, schwarz
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev, rel_err, STENCIL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


CASES = {
    "3d-ragged": lambda: syn.small_3d(24, 20, 12, seed=11),
    "3d-odd": lambda: syn.small_3d(17, 13, 9, seed=21),
    "2d-64": syn.config_small_2d,
}


def state_for(res, seed):
    p = syn.random_pressure(res, seed)
    rng = np.random.default_rng(seed)
    p_l = p * (1 - 0.02 * rng.random(p.size))
    p_lm1 = p_l * (1 - 0.02 * rng.random(p.size))
    return p, p_l, p_lm1


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("order", [1, 2])
def test_residual_and_jacobian(ras, case, order):
    res = CASES[case]()
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    p, p_l, p_lm1 = state_for(res, 5)
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, order, want_jac=True)
    Fd = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    nrm = gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, Fd, gp.J, want_norm=True)
    assert rel_err(host(Fd), F) < 1e-12
    for s, Jd in zip(STENCIL, gp.J):
        assert rel_err(host(Jd), J[s]) < 1e-12, s
    assert abs(nrm - np.linalg.norm(F)) <= 1e-12 * np.linalg.norm(F)
    # residual-only path agrees with the full one
    F2 = torch.zeros_like(Fd)
    gp.residual_eval(dev(p), dev(p_l), dev(p_lm1), res.dt, order, F2)
    assert torch.equal(F2, Fd)


def test_matvec(ras):
    res = CASES["3d-ragged"]()
    prob = disc.Problem(res)
    gp = ras.Problem(res)
    p, p_l, p_lm1 = state_for(res, 6)
    _, J = disc.residual(prob, p, p_l, p_lm1, res.dt, 2, want_jac=True)
    x = syn.random_vector(res.grid.n, 3)
    y = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.matvec(j_to_dev(J), dev(x), y)
    assert rel_err(host(y), disc.jacobian_csr(res.grid, J) @ x) < 1e-13


PARTS = [
    ("3d-ragged", (3, 2, 2), 1),
    ("3d-ragged", (4, 3, 2), 2),
    ("3d-ragged", (1, 1, 1), 1),   # one subdomain: global ILU(0)
    ("3d-ragged", (2, 2, 2), 0),   # delta = 0: block Jacobi with ILU(0)
    ("3d-odd", (3, 3, 2), 2),
    ("3d-odd", (17, 1, 1), 1),     # one-cell-wide owned slabs
    ("2d-64", (4, 4, 1), 1),
    ("2d-64", (5, 3, 1), 3),
]


def _jac(res, seed=7):
    prob = disc.Problem(res)
    p, p_l, p_lm1 = state_for(res, seed)
    _, J = disc.residual(prob, p, p_l, p_lm1, res.dt, 2, want_jac=True)
    return J, disc.jacobian_csr(res.grid, J)


@pytest.mark.parametrize("case,parts,overlap", PARTS)
def test_ras_apply_fp64(ras, case, parts, overlap):
    res = CASES[case]()
    J, A = _jac(res)
    g = res.grid
    M = schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, overlap)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, overlap, factor_prec=64)
    pc.factor(j_to_dev(J))
    for seed in (1, 2):
        r = syn.random_vector(g.n, seed)
        z = torch.full((g.n,), np.nan, dtype=torch.float64, device="cuda")
        pc.apply(dev(r), z)
        assert rel_err(host(z), M(r)) < 1e-12


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (16, 2e-2)])
@pytest.mark.parametrize("case,parts,overlap", [PARTS[1], PARTS[4], PARTS[6]])
def test_ras_apply_reduced_precision(ras, prec, tol, case, parts, overlap):
    res = CASES[case]()
    J, A = _jac(res)
    g = res.grid
    r = syn.random_vector(g.n, 4)
    emu = schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, overlap, prec=prec)(r)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, overlap, factor_prec=prec)
    pc.factor(j_to_dev(J))
    z = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), emu) < tol


def test_ras_apply_accumulates_nothing_between_calls(ras):
    res = CASES["3d-odd"]()
    J, A = _jac(res)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 2), 1, factor_prec=32)
    pc.factor(j_to_dev(J))
    r = dev(syn.random_vector(res.grid.n, 8))
    z1 = torch.zeros_like(r)
    z2 = torch.full_like(r, 1e30)
    pc.apply(r, z1)
    pc.apply(r, z2)
    assert torch.equal(z1, z2)  # deterministic, and every cell written


@pytest.mark.parametrize("restart", [30, 7])
def test_gmres_history_matches_oracle(ras, restart):
    """Newton-like system (BDF1 Jacobian at a smooth state). GMRES(30) converges
    in ~100 iterations over several restarts; GMRES(7) is stopped after 60
    iterations (it stagnates, which would amplify last-bit differences)."""
    res = CASES["3d-ragged"]()
    prob = disc.Problem(res)
    g = res.grid
    p0 = np.full(g.n, res.p0)
    p = syn.random_pressure(res, 9, 1.0, 3.0)
    F, J = disc.residual(prob, p, p0, p0, res.dt, 1, want_jac=True)
    A = disc.jacobian_csr(res.grid, J)
    parts, ov = (3, 2, 2), 1
    M = schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov)
    hist = []
    maxit = 500 if restart == 30 else 60
    x_ref, info = krylov.fgmres(lambda v: A @ v, M, -F, rtol=1e-8, atol=0.0, restart=restart,
                                maxit=maxit, history=hist)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=64)
    Jd = j_to_dev(J)
    pc.factor(Jd)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    out = gp.gmres_solve(Jd, pc, dev(-F), x, restart=restart, maxit=maxit, rtol=1e-8, atol=0.0)
    assert out["iters"] == info["iters"]
    h = np.array(out["history"])
    assert h.size == len(hist)
    hist = np.array(hist)
    rel = np.abs(h - hist) / np.abs(hist)
    detail = " ".join(f"{i}:{a:.6e}/{b:.6e}" for i, (a, b) in enumerate(zip(h, hist)) if rel[i] > 1e-10)
    # 1e-9 relative: of ||r0|| over the whole history, and of each entry down to the
    # FP64 floor of the Arnoldi residual estimate (~1e-11 ||r0|| here: entries that
    # small differ by rounding that the Givens recurrence carries from the start)
    assert np.max(np.abs(h - hist) / hist[0]) < 1e-9, detail
    assert np.all(np.abs(h - hist) <= 1e-9 * hist + 1e-11 * hist[0]), detail
    assert rel_err(host(x), x_ref) < 1e-9


def test_gmres_matches_dense_lu_tight(ras):
    res = syn.small_3d(8, 6, 4, seed=3)
    prob = disc.Problem(res)
    p, p_l, p_lm1 = state_for(res, 2)
    F, J = disc.residual(prob, p, p_l, p_lm1, res.dt, 2, want_jac=True)
    A = disc.jacobian_csr(res.grid, J).toarray()
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 1), 1)
    Jd = j_to_dev(J)
    pc.factor(Jd)
    x = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    gp.gmres_solve(Jd, pc, dev(-F), x, restart=30, maxit=300, rtol=1e-13)
    ref = np.linalg.solve(A, -F)
    assert rel_err(host(x), ref) < 1e-10


def _oracle_step(res, parts, ov, p_l, p_lm1, order, **kw):
    prob = disc.Problem(res)
    g = res.grid
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov)
    return newton.newton_solve(prob, fac, p_l, p_lm1, res.dt, order, **kw)


def test_newton_step_history_matches_oracle(ras):
    res = syn.config_small_2d()
    g = res.grid
    parts, ov = (4, 4, 1), 1
    p0 = np.full(g.n, res.p0)
    x_ref, info = _oracle_step(res, parts, ov, p0, p0, 1)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov)
    p = dev(p0)
    out = gp.newton_step(pc, p, dev(p0), dev(p0), res.dt, 1)
    assert out["status"] == 0
    assert out["newton_iters"] == info["newton_iters"]
    assert out["lin_iters"] == info["lin_iters"]
    assert np.allclose(out["lambdas"], info["lambdas"], rtol=1e-9)
    fh = np.array(out["fnorm_history"])
    ref = np.array(info["fnorm_history"])
    # 1e-9 relative, with the FP64 noise floor of ||F|| (~1e-13 ||F0||) allowed
    assert np.all(np.abs(fh - ref) <= 1e-9 * ref + 1e-12 * ref[0])
    assert rel_err(host(p), x_ref) < 1e-10


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_time_steps_match_oracle_state(ras, prec):
    """Five BDF steps (BDF1 then BDF2) of the 2D 64x64 workload."""
    res = syn.config_small_2d()
    g = res.grid
    parts, ov = (4, 4, 1), 1
    prob = disc.Problem(res)
    fac = lambda A, J: schwarz.Schwarz(A, (g.nx, g.ny, g.nz), parts, ov)
    states, infos = newton.simulate(prob, fac, 5)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, parts, ov, factor_prec=prec)
    p_l = dev(states[0])
    p_lm1 = p_l.clone()
    for step in range(5):
        p = p_l.clone()
        out = gp.newton_step(pc, p, p_l, p_lm1, res.dt, 1 if step == 0 else 2)
        assert out["status"] == 0
        assert rel_err(host(p), states[step + 1]) < (1e-10 if prec == 64 else 1e-6)
        if prec == 64:
            assert out["lin_iters"] == infos[step]["lin_iters"]
        p_lm1, p_l = p_l, p


def test_invalid_arguments_are_rejected(ras):
    res = CASES["3d-odd"]()
    gp = ras.Problem(res)
    with pytest.raises(ras.RasError) as e:
        ras.Precond(gp, (100, 1, 1), 1)          # more parts than cells
    assert e.value.status == ras.RAS_EINVAL
    with pytest.raises(ras.RasError):
        ras.Precond(gp, (2, 2, 2), 1, factor_prec=8)
    F = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    p = dev(np.full(res.grid.n, res.p0))
    with pytest.raises(ras.RasError):
        gp.residual_eval(p, p, p, -1.0, 1, F)      # negative dt
    with pytest.raises(ras.RasError):
        gp.residual_eval(p, p, p, 1.0, 3, F)       # unknown BDF order


def test_zero_pivot_reported(ras):
    res = syn.small_3d(6, 5, 4, seed=3)
    J, A = _jac(res)
    J["c"][0] = 0.0   # first cell of the first subdomain: zero pivot
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 1, 1), 1)
    with pytest.raises(ras.RasError) as e:
        pc.factor(j_to_dev(J))
    assert e.value.status == ras.RAS_EZEROPIVOT


def test_kernels_launch_through_the_library(ras):
    n0 = ras.kernel_launches()
    res = CASES["3d-odd"]()
    J, A = _jac(res)
    gp = ras.Problem(res)
    pc = ras.Precond(gp, (2, 2, 2), 1)
    pc.factor(j_to_dev(J))
    z = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
    pc.apply(dev(np.ones(res.grid.n)), z)
    assert ras.kernel_launches() > n0
