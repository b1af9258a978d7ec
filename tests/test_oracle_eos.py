"""Pins of the oracle's Peng-Robinson EOS (Section 2) against things it does not compute itself."""
import json
import os

import numpy as np
import pytest

from oracle import eos
from paper_2007_13966_gb300 import synthetic as syn

GOLD = os.path.join(os.path.dirname(__file__), "golden", "pr_methane.json")


def paper_fluid():
    return syn.Fluid.paper_methane()


def test_acentric_factor_from_paper_constants():
    g = json.load(open(GOLD))
    w = eos.acentric_factor(g["Tc"], g["pc"], g["Tb"])
    assert abs(w - g["omega_methane_expected"]) < g["omega_tolerance"]


def _np_roots_largest_real(A, B):
    r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
    real = r[np.abs(r.imag) < 1e-9 * max(1.0, np.abs(r).max())].real
    return real.max()


@pytest.mark.parametrize("fluid", [syn.Fluid(), syn.Fluid.paper_methane()])
def test_z_matches_companion_eigenvalues(fluid):
    a, b = eos.pr_constants(fluid)
    p = np.geomspace(1e3, 5e7, 60)
    Z = eos.z_factor(p, a, b, fluid.R, fluid.T)
    A, B = eos.AB(p, a, b, fluid.R, fluid.T)
    ref = np.array([_np_roots_largest_real(Ai, Bi) for Ai, Bi in zip(A, B)])
    assert np.max(np.abs(Z - ref) / ref) < 1e-12
    assert np.max(np.abs(eos.cubic(Z, A, B))) < 1e-14
    assert np.all(Z > B)


def test_z_tends_to_one_at_low_pressure():
    f = syn.Fluid()
    a, b = eos.pr_constants(f)
    Z = eos.z_factor(np.array([1e-2, 1.0, 1e2]), a, b, f.R, f.T)
    assert np.all(np.abs(Z - 1.0) < np.array([1e-9, 1e-6, 1e-4]))


def test_three_real_roots_takes_largest():
    # subcritical temperature: T < Tc gives three real roots near saturation
    f = syn.Fluid(T=150.0)
    a, b = eos.pr_constants(f)
    found = 0
    for p in np.linspace(5e5, 4e6, 200):
        A, B = eos.AB(p, a, b, f.R, f.T)
        r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        if np.all(np.abs(r.imag) < 1e-12):
            found += 1
            Z = eos.z_factor(np.array([p]), a, b, f.R, f.T)[0]
            assert abs(Z - r.real.max()) < 1e-10
            assert Z > np.sort(r.real)[1] + 1e-6
    assert found > 5


def test_ideal_gas_reduction():
    Z = eos.z_factor(np.array([1e5, 1e6]), 0.0, 0.0, 8.314, 300.0)
    assert np.all(Z == 1.0)


@pytest.mark.parametrize("fluid", [syn.Fluid(), syn.Fluid.paper_methane()])
def test_dz_dp_closed_form(fluid):
    a, b = eos.pr_constants(fluid)
    R, T = fluid.R, fluid.T
    p = np.geomspace(5e4, 3e7, 25)
    Z = eos.z_factor(p, a, b, R, T)
    d_paper = eos.dz_dp_paper(Z, p, a, b, R, T)
    d_impl = eos.dz_dp_implicit(Z, p, a, b, R, T)
    assert np.max(np.abs(d_paper - d_impl) / np.abs(d_impl)) < 1e-10
    h = 1e-4 * p
    fd = (eos.z_factor(p + h, a, b, R, T) - eos.z_factor(p - h, a, b, R, T)) / (2 * h)
    assert np.max(np.abs(d_paper - fd) / np.abs(fd)) < 1e-6


def test_d2z_dp2_finite_difference():
    f = syn.Fluid()
    a, b = eos.pr_constants(f)
    R, T = f.R, f.T
    p = np.geomspace(5e4, 3e7, 25)
    Z = eos.z_factor(p, a, b, R, T)
    dZ = eos.dz_dp_paper(Z, p, a, b, R, T)
    d2 = eos.d2z_dp2(Z, dZ, p, a, b, R, T)
    h = 1e-3 * p

    def dz(q):
        Zq = eos.z_factor(q, a, b, R, T)
        return eos.dz_dp_paper(Zq, q, a, b, R, T)
    fd = (dz(p + h) - dz(p - h)) / (2 * h)
    assert np.max(np.abs(d2 - fd) / np.abs(fd)) < 1e-5


def test_storage_and_mobility_derivatives():
    f = syn.Fluid()
    p = np.geomspace(5e4, 3e7, 20)
    Z, dZ, c, dc, m, dm = eos.eos_state(p, f)
    h = 1e-4 * p
    _, _, cp, _, mp, _ = eos.eos_state(p + h, f)
    _, _, cm, _, mm, _ = eos.eos_state(p - h, f)
    assert np.max(np.abs((cp - cm) / (2 * h) - dc) / np.abs(dc)) < 1e-5
    assert np.max(np.abs((mp - mm) / (2 * h) - dm) / np.abs(dm)) < 1e-7
    # density identity: c = d(p/Z)/dp (rho = p W / (Z R T), Eq. equ:density)
    rho_p = (p + h) / eos.eos_state(p + h, f)[0]
    rho_m = (p - h) / eos.eos_state(p - h, f)[0]
    assert np.max(np.abs((rho_p - rho_m) / (2 * h) - c) / c) < 1e-7


def test_m_branches():
    assert eos.m_of_omega(0.491) == pytest.approx(0.37464 + 1.54226 * 0.491 - 0.26992 * 0.491 ** 2)
    assert eos.m_of_omega(0.6) == pytest.approx(0.3796 + 1.485 * 0.6 - 0.1644 * 0.36 + 0.01667 * 0.216)
