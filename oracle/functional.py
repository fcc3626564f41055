"""Pointwise energy densities and potentials: Thomas-Fermi and Perdew-Zunger LDA (Sec. 2,
Sec. 3.3.1 of arXiv:1412.8250).

Oracle (test infrastructure only).  All functions take rho = u^2.  Pins
(tests/test_oracle_functional.py): uniform-gas closed forms (T_TF = C_F rho^{5/3} Omega,
E_x = -(3/4)(3/pi)^{1/3} rho^{4/3} Omega), V_TF and V_xc equal d(rho e)/d rho by a central
difference on both PZ branches, the branch split at r_s = 1, and continuity of e_c at
r_s = 1 to the rounding of the printed constants.
"""
from __future__ import annotations

from math import pi

import numpy as np

C_F = 0.3 * (3.0 * pi**2) ** (2.0 / 3.0)          # Eq. LR:KineticEnergy, C_F = (3/10)(3 pi^2)^{2/3}

# Perdew-Zunger constants as printed in Sec. 2
PZ = dict(gamma1=-0.1423, beta1=1.0529, beta2=0.3334, A1=0.0311, B1=-0.048, C1=0.002,
          D1=-0.0116)

RHO_FLOOR = 1e-24   # rho below this is treated as this value in the xc terms (u >= 1e-12)


def tf_energy_density(rho):
    """C_F u^{10/3} = C_F rho^{5/3} (Eq. TF:KineticEnergy)."""
    return C_F * np.asarray(rho) ** (5.0 / 3.0)


def tf_potential(rho):
    """V_TF = (5/3) C_F u^{4/3} (Sec. 3.3.1)."""
    return (5.0 / 3.0) * C_F * np.asarray(rho) ** (2.0 / 3.0)


def _rs(rho):
    return (3.0 / (4.0 * pi * np.maximum(rho, RHO_FLOOR))) ** (1.0 / 3.0)


def eps_xc(rho):
    """eps_x + eps_c per electron (Sec. 2): eps_x = -(3/4)(3/pi)^{1/3} u^{2/3}; eps_c the
    PZ form, first branch for r_s >= 1, logarithmic branch for r_s < 1."""
    rho = np.maximum(np.asarray(rho, dtype=float), RHO_FLOOR)
    ex = -0.75 * (3.0 / pi) ** (1.0 / 3.0) * rho ** (1.0 / 3.0)
    rs = _rs(rho)
    g, b1, b2 = PZ["gamma1"], PZ["beta1"], PZ["beta2"]
    A, B, C, D = PZ["A1"], PZ["B1"], PZ["C1"], PZ["D1"]
    ec_hi = g / (1.0 + b1 * np.sqrt(rs) + b2 * rs)
    ec_lo = A * np.log(rs) + B + C * rs * np.log(rs) + D * rs
    return ex + np.where(rs >= 1.0, ec_hi, ec_lo)


def xc_energy_density(rho):
    """eps_xc(u) u^2 (integrand of E_xc, Sec. 2)."""
    rho = np.asarray(rho, dtype=float)
    return eps_xc(rho) * np.maximum(rho, RHO_FLOOR)


def v_xc(rho):
    """V_xc = V_x + V_c (Sec. 3.3.1): V_x = -(3/pi)^{1/3} u^{2/3};
    V_c = (g + 7/6 g b1 sqrt(rs) + 4/3 g b2 rs) / (1 + b1 sqrt(rs) + b2 rs)^2 for r_s >= 1,
    V_c = (A + 2/3 C rs) ln rs + (B - A/3) + 1/3 (2D - C) rs for r_s < 1."""
    rho = np.maximum(np.asarray(rho, dtype=float), RHO_FLOOR)
    vx = -((3.0 / pi) ** (1.0 / 3.0)) * rho ** (1.0 / 3.0)
    rs = _rs(rho)
    g, b1, b2 = PZ["gamma1"], PZ["beta1"], PZ["beta2"]
    A, B, C, D = PZ["A1"], PZ["B1"], PZ["C1"], PZ["D1"]
    sq = np.sqrt(rs)
    vc_hi = (g + (7.0 / 6.0) * g * b1 * sq + (4.0 / 3.0) * g * b2 * rs) / (1.0 + b1 * sq + b2 * rs) ** 2
    vc_lo = (A + (2.0 / 3.0) * C * rs) * np.log(rs) + (B - A / 3.0) + (1.0 / 3.0) * (2.0 * D - C) * rs
    return vx + np.where(rs >= 1.0, vc_hi, vc_lo)
