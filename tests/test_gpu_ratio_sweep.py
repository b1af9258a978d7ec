"""Large coarse-to-fine ratios (Section 4's ratio study, Table 7: ratios 2 to 16 with
linear interpolation, Eq. equ:inter-second). At ratio r the support box of a coarse
basis function is 2r fine cells per axis, and from ratio 8 (FP64) or 16 (FP32) on in
3D the Galerkin product streams each term's box through shared memory in slabs of
fine planes instead of staging the seven terms' boxes whole. Checked here: the
exact coarse correction (Eq. equ:coarse-level) against the FP64 oracle at ratios
8 and 16 and an anisotropic (16, 8, 4), both coarse precisions; the slab form
gives the whole-box form's bits (slab height forced by RAS_RAP_SLAB); a support
that does not fit even one plane at a time is refused at set-up."""
import os

import numpy as np
import pytest
import torch

from oracle import discretization as disc
from oracle import multilevel as ml
from paper_2007_13966_gb300 import synthetic as syn

from gpu_util import dev, host, j_to_dev, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def _problem(dims, seed):
    res = syn.small_3d(*dims, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    return res, J, disc.jacobian_csr(res.grid, J)


def _precond(ras, gp, ratios, prec, env=None, parts=(2, 2, 2)):
    old = {k: os.environ.get(k) for k in (env or {})}
    os.environ.update(env or {})
    try:
        return ras.Precond(gp, parts, 1, nlevels=2, coarsen=ratios, mlevel_type=4, coarse_prec=prec)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


# (fine grid, ratios, subdomains): coarse 8 x 8 x 4 at ratio 8 (support 16 cells per
# axis), 4 x 4 x 2 at ratio 16 (32 cells: FP64 slabs of 14, 14 and 4 planes), and a
# per-axis mix; the subdomain counts keep every overlapped box within the fine
# solver's 16,384 cells (the coarse-only correction does not depend on them)
CASES = [((64, 64, 32), (8, 8, 8), (4, 4, 2)), ((64, 64, 32), (16, 16, 16), (4, 4, 2)),
         ((64, 48, 40), (16, 8, 4), (4, 4, 4))]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_large_ratio_coarse_correction_matches_oracle(ras, case, prec):
    dims, ratios, parts = CASES[case]
    res, J, A = _problem(dims, 11 + case)
    P = ml.interpolation(dims, ratios, 2)
    T = ml.TwoLevel(A, None, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.COARSE_ONLY)
    gp = ras.Problem(res)
    pc = _precond(ras, gp, ratios, prec, parts=parts)
    pc.factor(j_to_dev(J))
    r = syn.random_vector(res.grid.n, 3)
    z = torch.full((res.grid.n,), np.nan, dtype=torch.float64, device="cuda")
    pc.apply(dev(r), z)
    assert rel_err(host(z), T(r)) < (1e-9 if prec == 64 else 5e-3)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("dims,ratios,zs,parts", [
    ((24, 20, 28), (4, 4, 4), "3", (2, 2, 2)),     # support 8 planes: slabs of 3, 3, 2
    ((40, 24, 24), (2, 2, 2), "1", (2, 2, 2)),     # one plane at a time
    ((64, 64, 32), (8, 8, 8), "5", (4, 4, 2)),
])
def test_slab_form_has_the_whole_box_bits(ras, dims, ratios, zs, parts, prec):
    res, J, _ = _problem(dims, 7)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    r = dev(syn.random_vector(res.grid.n, 4))
    out = []
    for env in (None, {"RAS_RAP_SLAB": zs}):
        pc = _precond(ras, gp, ratios, prec, env, parts)
        pc.factor(Jd)
        z = torch.zeros_like(r)
        pc.apply(r, z)
        out.append(z)
        del pc
    assert torch.isfinite(out[0]).all()
    assert torch.equal(out[0], out[1])


def test_support_beyond_one_plane_slabs_is_refused(ras):
    """Ratio 32 across a 128 x 128 plane (FP64): interior supports of 64 x 64 cells
    per plane leave no room for even one plane beside the contraction buffers:
    RAS_EINVAL at set-up, before any launch."""
    res = syn.small_3d(128, 128, 4, seed=3)
    gp = ras.Problem(res)
    _precond(ras, gp, (16, 16, 1), 64)          # 32 x 32 supports: accepted
    with pytest.raises(ras.RasError):
        _precond(ras, gp, (32, 32, 1), 64)


def test_vcycle_fgmres_matches_oracle_across_ratios(ras):
    """FGMRES(30) to 1e-8 with the two-level V-cycle (FP64 factors and coarse LU) on a
    32 x 32 x 16 system at ratios 2, 4 and 8 (the last through the slab form): at every
    ratio the GPU takes the oracle's iterations (within one) along the same residual
    history, and the counts grow with the ratio as in Table 7."""
    from oracle import krylov, schwarz
    dims, parts = (32, 32, 16), (2, 2, 2)
    res = syn.small_3d(*dims, seed=9)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, 9)
    F, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, res.dt, 2, want_jac=True)
    A = disc.jacobian_csr(res.grid, J)
    M = schwarz.Schwarz(A, dims, parts, 1)
    gp = ras.Problem(res)
    Jd = j_to_dev(J)
    counts = []
    for r in (2, 4, 8):
        P = ml.interpolation(dims, (r, r, r), 2)
        T = ml.TwoLevel(A, M, P, ml.DenseCoarse(ml.galerkin(A, P)), ml.VCYCLE)
        hist = []
        x_ref, info = krylov.fgmres(lambda v: A @ v, T, -F, rtol=1e-8, atol=0.0, restart=30, maxit=500,
                                    history=hist)
        pc = ras.Precond(gp, parts, 1, factor_prec=64, nlevels=2, coarsen=(r, r, r), mlevel_type=0,
                         coarse_prec=64)
        pc.factor(Jd)
        x = torch.zeros(res.grid.n, dtype=torch.float64, device="cuda")
        out = gp.gmres_solve(Jd, pc, dev(-F), x, restart=30, maxit=500, rtol=1e-8, atol=0.0)
        assert abs(out["iters"] - info["iters"]) <= 1, (r, out["iters"], info["iters"])
        h = np.array(out["history"])
        m = min(h.size, len(hist))
        assert np.max(np.abs(h[:m] - np.array(hist[:m]))) <= 1e-8 * hist[0]
        assert rel_err(host(x), x_ref) < 1e-6
        counts.append(out["iters"])
        del pc
    assert counts == sorted(counts) and counts[0] < counts[-1], counts
