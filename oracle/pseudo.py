"""Charge density of the nuclei, self energy and overlap correction (Sec. 3.2, App. B).

Oracle (test infrastructure only).  The paper builds b_J = -(1/4pi) lap V_J from a tabulated
pseudopotential (Eq. b:Pseudopotential); those tables are not available, so every ion
carries a normalised Gaussian charge of width sigma, truncated at r_c:
    b_J(r) = -Z_J (2 pi sigma^2)^{-3/2} exp(-r^2 / (2 sigma^2)),   r <= r_c,
    V_J(r) = -Z_J erf(r / (sqrt(2) sigma)) / r        (so -(1/4pi) lap V_J = b_J).
b_J integrates to -Z_J (reading of the sign, so that u^2 + b is neutral, Sec. 3.3.1).

The overlap correction E_c^* of App. B is taken with point reference charges, for which the
b-b interaction of two Gaussians is Z_I Z_J erf(R/(2 sigma))/R in the continuum, giving
    E_c^* = 1/2 sum_I sum_{(J,T) != (I,0)} Z_I Z_J erfc(|R_I - R_J - T| / (2 sigma)) / |...|.

Pins (tests/test_oracle_pseudo.py): neutrality dV sum b = -sum Z; the Poisson potential of
b against the analytic periodic Fourier series; E_c^* against a brute-force direct lattice
sum with a larger cutoff; f^c against a central finite difference of E_c^*; the self energy
against its continuum value -(1/2) sum Z^2 / (sqrt(pi) sigma).
"""
from __future__ import annotations

from math import ceil, floor, pi, sqrt

import numpy as np
from scipy.special import erf, erfc

from .fd import Grid


def gaussian_b(r, Z, sigma):
    """Gaussian charge density of one ion, integrating to -Z (reading of Sec. 3.2)."""
    return -Z * (2.0 * pi * sigma**2) ** -1.5 * np.exp(-np.asarray(r) ** 2 / (2.0 * sigma**2))


def gaussian_V(r, Z, sigma):
    """Potential of that charge: -Z erf(r/(sqrt2 sigma))/r, limit -Z sqrt(2/pi)/sigma at 0."""
    r = np.asarray(r, dtype=float)
    out = np.empty_like(r)
    small = r < 1e-12
    out[~small] = -Z * erf(r[~small] / (sqrt(2.0) * sigma)) / r[~small]
    out[small] = -Z * sqrt(2.0 / pi) / sigma
    return out


def atom_box(R, rc, grid: Grid):
    """Unwrapped grid indices of the box enclosing the ball |x - R| <= rc.

    Returns (K, J, I) integer meshes (numpy order z, y, x) and the displacement arrays
    (DX, DY, DZ) = x - R.  Each unwrapped index is one periodic image of the ion: the
    point x = (i h1, j h2, k h3) maps to grid point (i mod n1, j mod n2, k mod n3)."""
    h = grid.h
    rng = [np.arange(ceil((R[d] - rc) / h[d]), floor((R[d] + rc) / h[d]) + 1) for d in range(3)]
    K, J, I = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    return (K, J, I), (I * h[0] - R[0], J * h[1] - R[1], K * h[2] - R[2])


def pseudocharge(R, Z, sigma, rc, grid: Grid) -> np.ndarray:
    """b(x) = sum_J sum_T b_J(|x - R_J - T|) over all images within r_c (Sec. 3.2, Sec. 4)."""
    b = np.zeros(grid.shape)
    n1, n2, n3 = grid.n
    for J in range(len(Z)):
        (K, Jj, I), (dx, dy, dz) = atom_box(R[J], rc, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        val = np.where(r <= rc, gaussian_b(r, Z[J], sigma), 0.0)
        np.add.at(b, (K % n3, Jj % n2, I % n1), val)
    return b


def pseudocharge_fd(R, Z, sigma, rc, grid: Grid):
    """The paper's construction b_J^{(i,j,k)} = -(1/4pi) (L_h V_J)^{(i,j,k)} (the nuclear charge
    of Sec. 4, from the pseudopotential by the same order-2N Laplacian as the rest), at the grid
    points within r_c of each image of ion J; V_J is sampled on the ion's box widened by N
    points each way so that every stencil tap is a sample.  Returns (b, e_self) with
    e_self = -(1/2) sum_J int b_J V_J over the same points."""
    from .fd import fd_laplacian_weights
    N = grid.N
    h = grid.h
    n1, n2, n3 = grid.n
    b = np.zeros(grid.shape)
    e = 0.0
    W = [fd_laplacian_weights(N, h[d]) for d in range(3)]
    for J in range(len(Z)):
        lo = [ceil((R[J][d] - rc) / h[d]) for d in range(3)]
        hi = [floor((R[J][d] + rc) / h[d]) for d in range(3)]
        ax = [np.arange(lo[d] - N, hi[d] + N + 1) * h[d] - R[J][d] for d in range(3)]
        DZ, DY, DX = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        V = gaussian_V(np.sqrt(DX**2 + DY**2 + DZ**2), Z[J], sigma)
        core = tuple(slice(N, -N) for _ in range(3))
        lap = np.zeros(V[core].shape)
        for d, axis in ((0, 2), (1, 1), (2, 0)):      # x is the last numpy axis
            for p in range(0, N + 1):
                sp = [slice(N, -N)] * 3
                sm = [slice(N, -N)] * 3
                m = V.shape[axis]
                sp[axis] = slice(N + p, m - N + p)
                sm[axis] = slice(N - p, m - N - p)
                lap += W[d][p] * (V[tuple(sp)] + V[tuple(sm)])
        r = np.sqrt(DX[core]**2 + DY[core]**2 + DZ[core]**2)
        bj = np.where(r <= rc, -lap / (4.0 * pi), 0.0)
        K, Jj, I = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                               np.arange(lo[0], hi[0] + 1), indexing="ij")
        np.add.at(b, (K % n3, Jj % n2, I % n1), bj)
        e += grid.dV * np.sum(bj * V[core])
    return b, -0.5 * e


def self_energy(R, Z, sigma, rc, grid: Grid) -> float:
    """Self-energy term -(1/2) sum_J int b_J V_J of Eq. LocalReformulationElectrostaticEnergy,
    each integral taken by the grid quadrature over the ion's support."""
    e = 0.0
    for J in range(len(Z)):
        _, (dx, dy, dz) = atom_box(R[J], rc, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        bj = np.where(r <= rc, gaussian_b(r, Z[J], sigma), 0.0)
        e += grid.dV * np.sum(bj * gaussian_V(r, Z[J], sigma))
    return -0.5 * e


def _image_range(L, cutoff):
    return [range(-int(ceil(cutoff / L[d])) - 1, int(ceil(cutoff / L[d])) + 2) for d in range(3)]


def repulsive_correction(R, Z, sigma, L, cutoff=None) -> float:
    """E_c^* for Gaussian charges with point reference charges (App. B, reading above)."""
    cutoff = 14.0 * sigma if cutoff is None else cutoff
    M = len(Z)
    e = 0.0
    for t1 in _image_range(L, cutoff)[0]:
        for t2 in _image_range(L, cutoff)[1]:
            for t3 in _image_range(L, cutoff)[2]:
                T = np.array([t1 * L[0], t2 * L[1], t3 * L[2]])
                for I in range(M):
                    for J in range(M):
                        if I == J and t1 == 0 and t2 == 0 and t3 == 0:
                            continue
                        r = np.linalg.norm(R[I] - R[J] - T)
                        if r <= cutoff:
                            e += 0.5 * Z[I] * Z[J] * erfc(r / (2.0 * sigma)) / r
    return float(e)


def repulsive_correction_forces(R, Z, sigma, L, cutoff=None) -> np.ndarray:
    """f^c_I = -dE_c^*/dR_I (App. B) for the closed form above."""
    cutoff = 14.0 * sigma if cutoff is None else cutoff
    M = len(Z)
    F = np.zeros((M, 3))
    for t1 in _image_range(L, cutoff)[0]:
        for t2 in _image_range(L, cutoff)[1]:
            for t3 in _image_range(L, cutoff)[2]:
                T = np.array([t1 * L[0], t2 * L[1], t3 * L[2]])
                for I in range(M):
                    for J in range(M):
                        if I == J and t1 == 0 and t2 == 0 and t3 == 0:
                            continue
                        d = R[I] - R[J] - T
                        r = np.linalg.norm(d)
                        if r <= cutoff:
                            # g(r) = erfc(r/2s)/r ; g'(r) = -exp(-r^2/4s^2)/(s sqrt(pi) r) - erfc/r^2
                            gp = (-np.exp(-r**2 / (4.0 * sigma**2)) / (sigma * sqrt(pi) * r)
                                  - erfc(r / (2.0 * sigma)) / r**2)
                            F[I] += -Z[I] * Z[J] * gp * d / r
    return F
