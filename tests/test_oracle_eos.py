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


MFIT = os.path.join(os.path.dirname(__file__), "golden", "pr_m_fit.json")


def _triple_root_constants():
    """Omega_a, Omega_b, Z_c of the Peng-Robinson critical point, solved here.

    At T = T_c and p = p_c the cubic of Eq. equ:PR has a triple root Z_c:
    matching Z^3 - (1-B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) with
    (Z - Z_c)^3 gives 3 Z_c = 1 - B, 3 Z_c^2 = A - 3B^2 - 2B and
    Z_c^3 = AB - B^2 - B^3, one equation in B after eliminating Z_c and A.
    """
    from scipy.optimize import brentq

    def g(B):
        Zc = (1.0 - B) / 3.0
        A = 3.0 * Zc * Zc + 3.0 * B * B + 2.0 * B
        return Zc ** 3 - (A * B - B * B - B ** 3)
    B = brentq(g, 0.01, 0.2, xtol=1e-16)
    Zc = (1.0 - B) / 3.0
    return 3.0 * Zc * Zc + 3.0 * B * B + 2.0 * B, B, Zc


@pytest.mark.parametrize("fluid", [syn.Fluid(), syn.Fluid.paper_methane()])
def test_pr_constants_at_the_critical_point(fluid):
    """a(T_c) p_c / (R T_c)^2 and b p_c / (R T_c) are the triple-root Omega_a, Omega_b
    to the digits Eq. attrfactor prints (half a unit of the last printed digit)."""
    Oa, Ob, Zc = _triple_root_constants()
    assert abs(Oa - 0.4572355) < 1e-7 and abs(Ob - 0.0777961) < 1e-7 and abs(Zc - 0.3074013) < 1e-7
    f = syn.Fluid(**{**fluid.__dict__, "T": fluid.Tc})
    a, b = eos.pr_constants(f)
    R, Tc, pc = f.R, f.Tc, f.pc
    assert abs(a * pc / (R * Tc) ** 2 - Oa) < 5e-6    # 0.45724: five decimals printed
    assert abs(b * pc / (R * Tc) - Ob) < 5e-5         # 0.0778: four decimals printed
    # the cubic at (T_c, p_c) with the printed constants has its roots near Z_c
    A, B = eos.AB(pc, a, b, R, Tc)
    r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
    assert np.max(np.abs(r - Zc)) < 0.03
    # and the oracle's root is the largest real one of them
    assert abs(eos.z_factor(np.array([pc]), a, b, R, Tc)[0] - r[np.abs(r.imag) < 1e-12].real.max()) < 1e-9


_S2 = float(np.sqrt(2.0))


def _ln_fugacity_coefficient(Z, A, B):
    """ln(f / p) of a Peng-Robinson phase with compressibility Z (the standard
    closed form of the integral of (Z - 1)/p at constant T)."""
    return (Z - 1.0 - np.log(Z - B)
            - A / (2.0 * _S2 * B) * np.log((Z + (1.0 + _S2) * B) / (Z + (1.0 - _S2) * B)))


def _saturation_pressure(a, b, R, T, pc):
    """Equal-fugacity pressure of the liquid (smallest) and vapour (largest) roots."""
    from scipy.optimize import brentq

    def g(p):
        A, B = a * p / (R * R * T * T), b * p / (R * T)
        r = np.roots([1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        re = np.sort(r[np.abs(r.imag) < 1e-10].real)
        if len(re) < 3:
            return None
        return _ln_fugacity_coefficient(re[-1], A, B) - _ln_fugacity_coefficient(re[0], A, B)
    grid = [(p, g(p)) for p in np.geomspace(1e-4 * pc, pc, 3000)]
    grid = [(p, v) for p, v in grid if v is not None]
    for (p0, v0), (p1, v1) in zip(grid, grid[1:]):
        if v0 * v1 < 0:
            return brentq(g, p0, p1, xtol=1e-13 * p0)
    raise AssertionError("no saturation pressure found")


@pytest.mark.parametrize("omega", [0.011, 0.2, 0.6])
def test_m_of_omega_reproduces_the_acentric_factor(omega):
    """The acentric factor is defined by log10(p_sat / p_c) = -(1 + omega) at
    T_r = 0.7; with m(omega) of Section 2 (and a(T) of Eq. attrfactor) the
    Peng-Robinson saturation pressure lands on that definition within the fit's
    accuracy (2.5e-3 in log10 on these points). omega = 0.6 takes the second
    branch; a wrong sign, a wrong power of T_r or a swapped branch fails."""
    f = syn.Fluid(T=0.7 * 190.6, omega=omega)
    a, b = eos.pr_constants(f)
    ps = _saturation_pressure(a, b, f.R, f.T, f.pc)
    assert abs(np.log10(ps / f.pc) + 1.0 + omega) < 4e-3


def test_m_branches_carry_the_printed_coefficients():
    """Coefficients recovered from m_of_omega by exact polynomial interpolation
    on each branch equal the ones Section 2 prints (tests/golden/pr_m_fit.json);
    at the shared end point 0.491 the first branch applies."""
    g = json.load(open(MFIT))
    for key, deg in (("m_low_branch", 2), ("m_high_branch", 3)):
        lo, hi = g[key]["range"]
        w = np.linspace(lo + 0.01, hi - 0.01, deg + 1)
        m = np.array([eos.m_of_omega(float(x)) for x in w])
        coef = np.linalg.solve(np.vander(w, deg + 1, increasing=True), m)
        assert np.allclose(coef, g[key]["coefficients_ascending"], rtol=0, atol=1e-9), (key, coef)
    c = g["m_low_branch"]["coefficients_ascending"]
    assert abs(eos.m_of_omega(0.491) - (c[0] + c[1] * 0.491 + c[2] * 0.491 ** 2)) < 1e-15
    # the a and b constants of Eq. attrfactor, as printed
    f = syn.Fluid(T=190.6)
    a, b = eos.pr_constants(f)
    assert abs(a * f.pc / (f.R * f.Tc) ** 2 - g["a_constant"]) < 1e-15
    assert abs(b * f.pc / (f.R * f.Tc) - g["b_constant"]) < 1e-15
