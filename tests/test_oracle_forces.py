"""Pins of the oracle's Hellmann-Feynman forces (Sec. 3.3.2, App. B)."""
from math import sqrt

import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W


def test_symmetric_fcc_cell_has_zero_forces():
    # ions on grid points of a perfect FCC cell: every ion sits at an inversion centre of
    # the grid and of b, so any potential built from b and a symmetric density exerts no force
    c = W.al4_cell(points_per_cell=16)
    grid = O.Grid(c.n, c.L, 6)
    b = O.pseudocharge(c.R, c.Z, c.sigma, c.rc, grid)
    u = np.full(grid.shape, sqrt(c.n_electrons / grid.volume))
    phi = O.poisson_solve(u * u + b, grid)
    F = O.forces(phi, c.R, c.Z, c.sigma, c.rc, grid)
    assert np.max(np.abs(F)) < 1e-10


def _ground_state_energy(cell, grid):
    res = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.tfw_functional(),
                             nlcg_tol=1e-7)
    return res


@pytest.mark.slow
def test_forces_match_energy_finite_difference():
    cell = W.small_cell(n=(16, 16, 16), sigma=1.0, rc=7.0, seed=21)
    grid = O.Grid(cell.n, cell.L, 6)
    res = _ground_state_energy(cell, grid)
    F = O.forces(res.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    d = 2e-3
    J, a = 1, 0
    E = []
    for sgn in (1, -1):
        c2 = W.small_cell(n=(16, 16, 16), sigma=1.0, rc=7.0, seed=21)
        c2.R[J, a] += sgn * d
        E.append(_ground_state_energy(c2, grid).energy)
    fd = -(E[0] - E[1]) / (2 * d)
    assert abs(fd - F[J, a]) < 1e-6
    # momentum balance: the forces sum to ~0 (broken only by the grid)
    assert np.max(np.abs(F.sum(0))) < 1e-7
