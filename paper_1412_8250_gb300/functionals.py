"""Kinetic functionals of Eq. KineticEnergyComponents as of_functional records.

TFW: lambda = 1/5, mu = 0 (the paper's TFW choice, Sec. 5).
WT-type: lambda = mu = 1 with the density-independent m = n = 0 kernel term, exponents
alpha, beta = (5 +- sqrt5)/6 and the R = 4 rational fit of App. A (Table ConstantsHelmholtz,
rows P_00r and Q_00r; r = 2, 4 are the complex conjugates of r = 1, 3).
WGC: the same with the second-order expansion of the density-dependent kernel (L = 2, Sec. 5),
rows P_10r ... Q_11r of the same table.
"""
from math import pi, sqrt

from . import binding as B

# App. A, Table ConstantsHelmholtz: P_00r, Q_00r for r = 1 and r = 3
P00 = (0.108403 + 0.079657j, -0.908403 + 0.439708j)
Q00 = (-0.470923 - 0.465392j, 0.066051 - 0.259678j)


def tfw(lam=0.2):
    return B.make_functional(lam, 0.0)


# rows (m, n) = (1, 0), (2, 0), (1, 1): (P_r, Q_r) for r = 1 and r = 3
WGC_ROWS = {
    "10": ((-0.030515 + 0.015027j, 0.028915 - 0.008817j),
           (-0.597793 - 0.294130j, -0.087917 - 0.164937j)),
    "20": ((0.008907 - 0.032841j, -0.034974 + 0.009116j),
           (-0.537986 - 0.233840j, -0.041565 - 0.196662j)),
    "11": ((0.012423 - 0.034421j, -0.031907 + 0.007392j),
           (-0.511699 - 0.0266195j, -0.034031 - 0.188927j)),
}


def _pairs(v):
    return (v[0], v[0].conjugate(), v[1], v[1].conjugate())


def wt():
    return B.make_functional(1.0, 1.0, (5.0 + sqrt(5.0)) / 6.0, (5.0 - sqrt(5.0)) / 6.0,
                             _pairs(P00), _pairs(Q00))


def wgc():
    K = {c: (_pairs(P), _pairs(Q)) for c, (P, Q) in WGC_ROWS.items()}
    return B.make_functional(1.0, 1.0, (5.0 + sqrt(5.0)) / 6.0, (5.0 - sqrt(5.0)) / 6.0,
                             _pairs(P00), _pairs(Q00), L=2, K=K)


def kf2(n_electrons, volume):
    """(2 kF)^2 with kF = (3 pi^2 N_e / Omega)^{1/3} (Sec. 3.1)."""
    kf = (3.0 * pi * pi * n_electrons / volume) ** (1.0 / 3.0)
    return 4.0 * kf * kf
