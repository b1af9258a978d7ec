"""Peng-Robinson equation of state, Section 2 (oracle; test infrastructure only).

Notation follows Section 2: A = a p / (R^2 T^2), B = b p / (R T), the PR cubic
Z^3 - (1-B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0 (Eq. equ:PR),
a(T), b from the critical point (Eq. attrfactor), m(omega) with two branches,
omega from the reduced normal boiling point, and the closed form of dZ/dp
printed under Eq. gover_sys.

Readings where the paper is silent or garbled:
* Eq. attrfactor's sentence swaps the words "pressure"/"temperature" for T_c and
  p_c; T_c is read as the critical temperature and p_c as the critical pressure.
* At omega = 0.491 both m branches apply; the first (quadratic) one is used.
* Root selection is deferred to the paper's references: the largest real root
  (the vapour root) is taken; it is computed in closed form (Cardano /
  trigonometric) and polished by two Newton steps on the cubic.
* d2Z/dp2 (needed for the exact Jacobian of the accumulation term) is obtained
  by differentiating the cubic relation twice.
"""
from __future__ import annotations

import math

import numpy as np

ATM = 101325.0


def acentric_factor(Tc: float, pc: float, Tb: float) -> float:
    """omega = (-ln(p_c / 1 atm) - f0(T_br)) / f1(T_br), T_br = T_b / T_c (Section 2)."""
    Tbr = Tb / Tc
    tau = 1.0 - Tbr
    f0 = (-5.97616 * tau + 1.29874 * tau ** 1.5 - 0.60394 * tau ** 2.5
          - 1.06841 * tau ** 5) / Tbr
    f1 = (-5.03365 * tau + 1.11505 * tau ** 1.5 - 5.41217 * tau ** 2.5
          - 7.46628 * tau ** 5) / Tbr
    return (-math.log(pc / ATM) - f0) / f1


def m_of_omega(w: float) -> float:
    """The two-branch fit of m in the acentric factor (Section 2)."""
    if w <= 0.491:
        return 0.37464 + 1.54226 * w - 0.26992 * w * w
    return 0.3796 + 1.485 * w - 0.1644 * w * w + 0.01667 * w ** 3


def pr_constants(fluid):
    """(a, b) of Eq. attrfactor for the fluid at its temperature T."""
    omega = acentric_factor(fluid.Tc, fluid.pc, fluid.Tb) if fluid.omega_from_Tb else fluid.omega
    m = m_of_omega(omega)
    R, T, Tc, pc = fluid.R, fluid.T, fluid.Tc, fluid.pc
    a = 0.45724 * R * R * Tc * Tc / pc * (1.0 + m * (1.0 - math.sqrt(T / Tc))) ** 2
    b = 0.0778 * R * Tc / pc
    return a, b


def AB(p, a, b, R, T):
    """A = a p / (R^2 T^2), B = b p / (R T)."""
    return a * p / (R * R * T * T), b * p / (R * T)


def cubic(Z, A, B):
    """Left-hand side of Eq. equ:PR."""
    return Z ** 3 - (1.0 - B) * Z ** 2 + (A - 3.0 * B ** 2 - 2.0 * B) * Z - (A * B - B ** 2 - B ** 3)


def cubic_dZ(Z, A, B):
    """C = 3Z^2 - 2(1-B)Z + (A - 2B - 3B^2), the Z-derivative of the cubic."""
    return 3.0 * Z ** 2 - 2.0 * (1.0 - B) * Z + (A - 2.0 * B - 3.0 * B ** 2)


def largest_real_root(c2, c1, c0):
    """Largest real root of Z^3 + c2 Z^2 + c1 Z + c0 = 0 (closed form).

    Depressed cubic Z = t - c2/3: t^3 + P t + Q = 0. One real root (Cardano)
    when the discriminant Q^2/4 + P^3/27 > 0, three real roots otherwise
    (trigonometric form, k = 0 branch is the largest).
    """
    c2 = np.asarray(c2, dtype=np.float64)
    c1 = np.asarray(c1, dtype=np.float64)
    c0 = np.asarray(c0, dtype=np.float64)
    P = c1 - c2 * c2 / 3.0
    Q = 2.0 * c2 ** 3 / 27.0 - c2 * c1 / 3.0 + c0
    disc = Q * Q / 4.0 + P ** 3 / 27.0
    out = np.empty_like(P)
    one = disc > 0
    s = np.sqrt(np.where(one, disc, 0.0))
    u = np.cbrt(-Q / 2.0 + s)
    v = np.cbrt(-Q / 2.0 - s)
    out[one] = (u + v)[one]
    three = ~one
    if np.any(three):
        Pm = np.minimum(P[three], 0.0)
        r = np.sqrt(-Pm / 3.0)
        arg = np.where(r > 0, (-Q[three] / 2.0) / np.where(r > 0, r ** 3, 1.0), 0.0)
        arg = np.clip(arg, -1.0, 1.0)
        out[three] = 2.0 * r * np.cos(np.arccos(arg) / 3.0)
    return out - c2 / 3.0


def z_factor(p, a, b, R, T, polish: int = 2):
    """Compressibility factor Z(p): largest real root of Eq. equ:PR, Newton-polished."""
    p = np.asarray(p, dtype=np.float64)
    A, B = AB(p, a, b, R, T)
    c2 = -(1.0 - B)
    c1 = A - 3.0 * B ** 2 - 2.0 * B
    c0 = -(A * B - B ** 2 - B ** 3)
    Z = largest_real_root(c2, c1, c0)
    for _ in range(polish):
        Z = Z - cubic(Z, A, B) / cubic_dZ(Z, A, B)
    return Z


def dz_dp_paper(Z, p, a, b, R, T):
    """dZ/dp, the closed form printed under Eq. gover_sys."""
    A, B = AB(p, a, b, R, T)
    C = cubic_dZ(Z, A, B)
    RT = R * T
    return (-(b / (RT * C)) * Z ** 2
            - (a / (RT * RT * C) - (2.0 * b + 6.0 * B * b) / (RT * C)) * Z
            + (2.0 * a * b * p / (RT ** 3 * C) - (2.0 * B * b + 3.0 * B * B * b) / (RT * C)))


def _partials(Z, p, a, b, R, T):
    """Partial derivatives of f(Z, p) = cubic with A = alpha p, B = beta p."""
    al = a / (R * R * T * T)
    be = b / (R * T)
    fZ = 3 * Z ** 2 - 2 * (1 - be * p) * Z + (al * p - 3 * be ** 2 * p ** 2 - 2 * be * p)
    fp = be * Z ** 2 + (al - 6 * be ** 2 * p - 2 * be) * Z - (2 * al * be * p - 2 * be ** 2 * p - 3 * be ** 3 * p ** 2)
    fZZ = 6 * Z - 2 * (1 - be * p)
    fZp = 2 * be * Z + (al - 6 * be ** 2 * p - 2 * be)
    fpp = -6 * be ** 2 * Z - (2 * al * be - 2 * be ** 2 - 6 * be ** 3 * p)
    return fZ, fp, fZZ, fZp, fpp


def dz_dp_implicit(Z, p, a, b, R, T):
    """dZ/dp = -f_p / f_Z from implicit differentiation of the cubic."""
    fZ, fp, *_ = _partials(Z, p, a, b, R, T)
    return -fp / fZ


def d2z_dp2(Z, dZ, p, a, b, R, T):
    """d2Z/dp2 = -(f_ZZ Z'^2 + 2 f_Zp Z' + f_pp) / f_Z."""
    fZ, _, fZZ, fZp, fpp = _partials(Z, p, a, b, R, T)
    return -(fZZ * dZ * dZ + 2.0 * fZp * dZ + fpp) / fZ


def eos_state(p, fluid, a=None, b=None):
    """Per-cell EOS quantities used by the residual.

    Returns (Z, dZ, c, dc, m, dm) where, following Eq. gover_sys,
    c = (p/Z)(1/p - Z'/Z) is the storage coefficient and m = p / (mu Z) the
    mobility-density factor of the flux; dc, dm are their p-derivatives.
    """
    if a is None:
        a, b = pr_constants(fluid)
    R, T, mu = fluid.R, fluid.T, fluid.mu
    p = np.asarray(p, dtype=np.float64)
    Z = z_factor(p, a, b, R, T)
    dZ = dz_dp_paper(Z, p, a, b, R, T)
    d2Z = d2z_dp2(Z, dZ, p, a, b, R, T)
    c = (p / Z) * (1.0 / p - dZ / Z)
    # dc/dp of c = 1/Z - p Z'/Z^2
    dc = -2.0 * dZ / Z ** 2 - p * d2Z / Z ** 2 + 2.0 * p * dZ * dZ / Z ** 3
    m = p / (mu * Z)
    dm = c / mu
    return Z, dZ, c, dc, m, dm
