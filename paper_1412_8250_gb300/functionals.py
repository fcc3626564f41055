"""Kinetic functionals of Eq. KineticEnergyComponents as of_functional records.

TFW: lambda = 1/5, mu = 0 (the paper's TFW choice, Sec. 5).
WT-type: lambda = mu = 1 with the density-independent m = n = 0 kernel term, exponents
alpha, beta = (5 +- sqrt5)/6 and the R = 4 rational fit of App. A (Table ConstantsHelmholtz,
rows P_00r and Q_00r; r = 2, 4 are the complex conjugates of r = 1, 3).
"""
from math import pi, sqrt

from . import binding as B

# App. A, Table ConstantsHelmholtz: P_00r, Q_00r for r = 1 and r = 3
P00 = (0.108403 + 0.079657j, -0.908403 + 0.439708j)
Q00 = (-0.470923 - 0.465392j, 0.066051 - 0.259678j)


def tfw(lam=0.2):
    return B.make_functional(lam, 0.0)


def wt():
    P = (P00[0], P00[0].conjugate(), P00[1], P00[1].conjugate())
    Q = (Q00[0], Q00[0].conjugate(), Q00[1], Q00[1].conjugate())
    return B.make_functional(1.0, 1.0, (5.0 + sqrt(5.0)) / 6.0, (5.0 - sqrt(5.0)) / 6.0, P, Q)


def kf2(n_electrons, volume):
    """(2 kF)^2 with kF = (3 pi^2 N_e / Omega)^{1/3} (Sec. 3.1)."""
    kf = (3.0 * pi * pi * n_electrons / volume) ** (1.0 / 3.0)
    return 4.0 * kf * kf
