"""Pins of the oracle's discrete adjoint (oracle/adjoint.py): the gradient of
the producer-pressure objective agrees with central finite differences of the
oracle's own time loop, on 2D and 3D grids and for BDF1-only and BDF2 runs."""
import numpy as np
import pytest

from oracle import adjoint as adj
from paper_2007_13966_gb300 import synthetic as syn


def small(dims, seed):
    nx, ny, nz = dims
    if nz == 1:
        return syn.lognormal_reservoir(nx, ny, 1, 20.0, 20.0, 1.0, sigma=1.0, corr=2.0,
                                       seed_k=seed, seed_phi=seed + 1)
    return syn.small_3d(nx, ny, nz, seed=seed)


@pytest.mark.parametrize("dims,nsteps", [((6, 5, 3), 3), ((7, 6, 1), 4), ((5, 4, 2), 1)])
def test_adjoint_gradient_matches_finite_differences(dims, nsteps):
    res = small(dims, 3)
    cells = adj.producer_cells(res)
    phi, grad, lam = adj.adjoint_gradient(res, nsteps, cells)
    n = res.grid.n
    rng = np.random.default_rng(1)
    idx = list(cells[:1]) + [0, n - 1] + list(rng.choice(n, 4, replace=False))
    fd = adj.fd_gradient(res, nsteps, cells, idx, h=1e-5)
    scale = np.abs(grad).max()
    assert scale > 0
    assert np.abs(grad[idx] - fd).max() <= 2e-5 * scale


def test_objective_and_adjoint_shapes():
    res = small((5, 4, 2), 4)
    cells = adj.producer_cells(res)
    assert cells.size == 2                       # the producer column of a 2-layer grid
    phi, grad, lam = adj.adjoint_gradient(res, 2, cells)
    assert phi > 0 and grad.shape == (res.grid.n,) and len(lam) == 2


def test_perturbation_scales_connections():
    res = small((5, 4, 2), 5)
    th = np.linspace(-0.5, 0.5, res.grid.n)
    r2 = adj.perturbed(res, th)
    e = np.exp(th)
    assert np.allclose(r2.kx, res.kx * e, rtol=1e-14, atol=0)
    assert np.allclose(r2.kz, res.kz * e, rtol=1e-14, atol=0)
    assert np.allclose(r2.conns.T, res.conns.T * e[res.conns.cell], rtol=1e-14, atol=0)


@pytest.mark.parametrize("options", [{"conservative": True}, {"gravity": 50 * 9.80665, "upwind": True}])
def test_adjoint_gradient_with_physics_options(options):
    """The same pin with the conservative accumulation form (whose time-level
    coupling takes c at the older state) and with gravity plus upstream mobility,
    at 30-300 atm, where the gas is far enough from ideal for c to differ between
    time levels."""
    import dataclasses
    base = small((6, 5, 3), 3)
    c = base.conns
    res = dataclasses.replace(base, conns=syn.Connections(c.cell.copy(), 30 * c.p, c.T.copy()),
                              p0=30 * syn.ATM, **options)
    cells = adj.producer_cells(res)
    phi, grad, lam = adj.adjoint_gradient(res, 3, cells)
    n = res.grid.n
    idx = list(cells[:1]) + [0, n - 1] + list(np.random.default_rng(2).choice(n, 4, replace=False))
    fd = adj.fd_gradient(res, 3, cells, idx, h=1e-5)
    scale = np.abs(grad).max()
    assert scale > 0
    assert np.abs(grad[idx] - fd).max() <= 1e-7 * scale
