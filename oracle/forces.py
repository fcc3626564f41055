"""Hellmann-Feynman forces on the nuclei (Sec. 3.3.2, Eq. Force:Nuclei; App. B for f^c).

Oracle (test infrastructure only).  f_J = sum over J and its periodic images of
int grad b_J (phi* - V_J) dx + f_J^c, the integral taken by the grid quadrature over the
ball of radius r_c around each image, grad b_J the analytic gradient of the Gaussian charge
(grad b_J(x) = -b_J(x) (x - R_J) / sigma^2).

Pins (tests/test_oracle_forces.py): zero forces for a symmetric FCC cell on the grid; the
central finite difference of the ground-state energy with respect to an ion position; the
closed-form f^c against finite differences of E_c^*.
"""
from __future__ import annotations

import numpy as np

from .fd import Grid
from .pseudo import atom_box, gaussian_b, gaussian_V, repulsive_correction_forces


def forces(phi, R, Z, sigma, rc, grid: Grid, include_correction=True) -> np.ndarray:
    n1, n2, n3 = grid.n
    M = len(Z)
    F = np.zeros((M, 3))
    for J in range(M):
        (K, Jj, I), (dx, dy, dz) = atom_box(R[J], rc, grid)
        r = np.sqrt(dx**2 + dy**2 + dz**2)
        inside = r <= rc
        bJ = np.where(inside, gaussian_b(r, Z[J], sigma), 0.0)
        w = phi[K % n3, Jj % n2, I % n1] - gaussian_V(r, Z[J], sigma)
        for c, dc in enumerate((dx, dy, dz)):
            F[J, c] = grid.dV * np.sum(-bJ * dc / sigma**2 * w)
    if include_correction:
        F += repulsive_correction_forces(R, Z, sigma, grid.L)
    return F
