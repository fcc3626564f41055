"""The overlap correction E_c^* evaluated on the grid with reference charges (App. B,
Eq. RepulsiveCorrection2 and the force expression f_J^c that follows it).

Oracle (test infrastructure only).  The reference charges are Gaussians of a narrower width
sigma_ref, b~_J(r) = -Z_J (2 pi sigma_ref^2)^{-3/2} exp(-r^2 / 2 sigma_ref^2) for
r <= rc_ref (the same sign convention as b_J, so that b~ - b is neutral), with potentials
V~_J = -Z_J erf(r / (sqrt2 sigma_ref)) / r.  Then

    E_c^* = 1/2 int (b~ + b) V_c + 1/2 sum_J int b_J V_J - 1/2 sum_J int b~_J V~_J,
    -(1/4 pi) L_h V_c = b~ - b,

every integral the grid quadrature, the self integrals over each ion's support.  V_c is fixed
up to a constant by the periodic solve; the constant is set so that V_c at the grid point
x0 = 0 equals sum_J (V~_J - V_J)(x0), the sum over the ions and their periodic images (App. B
says to evaluate that sum at any point; the sign follows from -(1/4 pi) Lap (V~_J - V_J) =
b~_J - b_J).

Forces (the printed second form, J' running over ion J and its periodic images):

    f_J^c = 1/2 sum_J' int [ grad b~_J' (V_c - V~_J') + grad b_J' (V_c + V_J')
                             + grad V_c,J' (b~ + b) + b_J' grad V_J' - b~_J' grad V~_J' ],

with V_c,J' = V~_J' - V_J'.  Each term is integrated over the ball where its compactly
supported factor lives (r_c for b, rc_ref for b~) and, for grad V_c,J' (b~ + b), over the ball
of radius `cutoff` beyond which V~_J - V_J is below rounding (it decays like erfc(r/sqrt2 sigma)).

Pins (tests/test_oracle_overlap.py): with sigma_ref = sigma the correction and its forces
vanish; with non-overlapping reference charges E_c^* converges, as h -> 0, to the pair sum
1/2 sum_{I != J} Z_I Z_J [erfc(R/2 sigma) - erfc(R/2 sigma_ref)] / R (a real-space route that
shares nothing with the grid solve), and so do the forces to that sum's derivative; the forces
agree with central differences of this grid energy and sum to zero.
"""
from __future__ import annotations

from math import ceil, pi, sqrt

import numpy as np
from scipy.special import erf, erfc

from .fd import Grid, poisson_solve
from .pseudo import atom_box, gaussian_b, gaussian_V, pseudocharge, self_energy


def gaussian_grad_V(dx, dy, dz, Z, sigma):
    """Gradient (with respect to x) of V_J = -Z erf(r / (sqrt2 sigma)) / r at x - R_J = d."""
    r = np.sqrt(dx**2 + dy**2 + dz**2)
    out = np.zeros((3,) + np.shape(r))
    ok = r > 1e-12
    ro = r[ok]
    # dV/dr = -Z [ sqrt(2/pi)/sigma exp(-r^2/2sigma^2) / r - erf(r/(sqrt2 sigma)) / r^2 ]
    dVdr = -Z * (sqrt(2.0 / pi) / sigma * np.exp(-ro**2 / (2.0 * sigma**2)) / ro
                 - erf(ro / (sqrt(2.0) * sigma)) / ro**2)
    for c, dc in enumerate((dx, dy, dz)):
        out[c][ok] = dVdr * dc[ok] / ro
    return out


def potential_difference_at(x0, R, Z, sigma, sigma_ref, L, cutoff):
    """sum over ions J and images T of (V~_J - V_J)(|x0 - R_J - T|), terms beyond `cutoff`
    dropped (their size is ~ Z erfc(cutoff / (sqrt2 max(sigma, sigma_ref))) / cutoff)."""
    s = 0.0
    reps = [int(ceil(cutoff / L[d])) + 1 for d in range(3)]
    for J in range(len(Z)):
        for t1 in range(-reps[0], reps[0] + 1):
            for t2 in range(-reps[1], reps[1] + 1):
                for t3 in range(-reps[2], reps[2] + 1):
                    d = np.asarray(x0) - R[J] - np.array([t1 * L[0], t2 * L[1], t3 * L[2]])
                    r = np.array([np.linalg.norm(d)])
                    if r[0] <= cutoff:
                        s += float(gaussian_V(r, Z[J], sigma_ref)[0] - gaussian_V(r, Z[J], sigma)[0])
    return s


def repulsive_correction_grid(R, Z, sigma, rc, sigma_ref, rc_ref, grid: Grid, cutoff=None):
    """E_c^* of Eq. RepulsiveCorrection2 on the grid; returns (E_c^*, V_c, b~ + b)."""
    R = np.asarray(R, dtype=float)
    cutoff = 12.0 * max(sigma, sigma_ref) if cutoff is None else cutoff
    b = pseudocharge(R, Z, sigma, rc, grid)
    bt = pseudocharge(R, Z, sigma_ref, rc_ref, grid)
    Vc = poisson_solve(bt - b, grid)
    Vc = Vc + (potential_difference_at((0.0, 0.0, 0.0), R, Z, sigma, sigma_ref, grid.L, cutoff)
               - Vc[0, 0, 0])
    E = (0.5 * grid.dV * float(np.sum((bt + b) * Vc))
         - self_energy(R, Z, sigma, rc, grid)            # + 1/2 sum_J int b_J V_J
         + self_energy(R, Z, sigma_ref, rc_ref, grid))   # - 1/2 sum_J int b~_J V~_J
    return E, Vc, bt + b


def repulsive_correction_grid_forces(R, Z, sigma, rc, sigma_ref, rc_ref, grid: Grid,
                                     cutoff=None):
    """f_J^c of App. B on the grid (the expression in the module header)."""
    R = np.asarray(R, dtype=float)
    cutoff = 12.0 * max(sigma, sigma_ref) if cutoff is None else cutoff
    _, Vc, bsum = repulsive_correction_grid(R, Z, sigma, rc, sigma_ref, rc_ref, grid, cutoff)
    n1, n2, n3 = grid.n
    M = len(Z)
    F = np.zeros((M, 3))
    for J in range(M):
        # grad b_J' (V_c + V_J') + b_J' grad V_J' over the balls r <= rc
        (K, Jj, I), (dx, dy, dz) = atom_box(R[J], rc, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        inside = r <= rc
        bJ = np.where(inside, gaussian_b(r, Z[J], sigma), 0.0)
        vc = Vc[K % n3, Jj % n2, I % n1]
        gV = gaussian_grad_V(dx, dy, dz, Z[J], sigma)
        for c, dc in enumerate((dx, dy, dz)):
            grad_b = -bJ * dc / sigma**2
            F[J, c] += 0.5 * grid.dV * np.sum(grad_b * (vc + gaussian_V(r, Z[J], sigma)) + bJ * gV[c])
        # grad b~_J' (V_c - V~_J') - b~_J' grad V~_J' over the balls r <= rc_ref
        (K, Jj, I), (dx, dy, dz) = atom_box(R[J], rc_ref, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        inside = r <= rc_ref
        bJ = np.where(inside, gaussian_b(r, Z[J], sigma_ref), 0.0)
        vc = Vc[K % n3, Jj % n2, I % n1]
        gV = gaussian_grad_V(dx, dy, dz, Z[J], sigma_ref)
        for c, dc in enumerate((dx, dy, dz)):
            grad_b = -bJ * dc / sigma_ref**2
            F[J, c] += 0.5 * grid.dV * np.sum(grad_b * (vc - gaussian_V(r, Z[J], sigma_ref))
                                              - bJ * gV[c])
        # grad V_c,J' (b~ + b) over the balls r <= cutoff
        (K, Jj, I), (dx, dy, dz) = atom_box(R[J], cutoff, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        inside = r <= cutoff
        w = np.where(inside, bsum[K % n3, Jj % n2, I % n1], 0.0)
        gVc = gaussian_grad_V(dx, dy, dz, Z[J], sigma_ref) - gaussian_grad_V(dx, dy, dz, Z[J], sigma)
        for c in range(3):
            F[J, c] += 0.5 * grid.dV * np.sum(gVc[c] * w)
    return F


def repulsive_correction_pairs(R, Z, sigma, sigma_ref, L, cutoff=None) -> float:
    """The continuum value of the same correction for Gaussian b and b~: two Gaussians of
    widths s_a, s_b at distance R interact as Z_I Z_J erf(R / sqrt(2 (s_a^2 + s_b^2))) / R, so
    E_c^* = 1/2 sum_{I != J (images included)} Z_I Z_J [erfc(R/2 sigma) - erfc(R/2 sigma_ref)] / R."""
    R = np.asarray(R, dtype=float)
    cutoff = 14.0 * max(sigma, sigma_ref) if cutoff is None else cutoff
    reps = [int(ceil(cutoff / L[d])) + 1 for d in range(3)]
    e = 0.0
    M = len(Z)
    for t1 in range(-reps[0], reps[0] + 1):
        for t2 in range(-reps[1], reps[1] + 1):
            for t3 in range(-reps[2], reps[2] + 1):
                T = np.array([t1 * L[0], t2 * L[1], t3 * L[2]])
                for I in range(M):
                    for J in range(M):
                        if I == J and t1 == 0 and t2 == 0 and t3 == 0:
                            continue
                        r = float(np.linalg.norm(R[I] - R[J] - T))
                        if r <= cutoff:
                            e += 0.5 * Z[I] * Z[J] * (erfc(r / (2.0 * sigma))
                                                      - erfc(r / (2.0 * sigma_ref))) / r
    return e
