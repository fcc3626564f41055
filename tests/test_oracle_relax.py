"""Pins of the oracle's geometry relaxation (Sec. 3.3: NLCG on the nuclear positions with the
Polak-Ribiere update and a secant line search on the forces)."""
import numpy as np

import oracle as O
from oracle.relax import relax
from paper_1412_8250_gb300 import workloads as W


def test_displaced_atom_returns_to_the_perfect_lattice():
    # the perfect FCC cell is a stationary point by symmetry; from one atom moved by 0.25 bohr
    # the relaxation must come back to it, up to the common translation (the forces sum to
    # zero, so the centre of the cell moves by 0.25 / 4)
    cell = W.al4_cell(points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    R0 = cell.R.copy()
    R0[0, 0] += 0.25
    r = relax(grid, R0, cell.Z, cell.sigma, cell.rc, O.tfw_functional(), ftol=1e-5, nlcg_tol=1e-9)
    assert r.max_force < 1e-5
    rel = (r.R - r.R[0]) - (cell.R - cell.R[0])
    assert np.abs(rel).max() < 1e-3
    shift = r.R.mean(axis=0) - R0.mean(axis=0)
    assert np.abs(shift).max() < 2e-3          # momentum balance: the centre barely moves
    # every accepted step lowers the energy
    assert all(b < a + 1e-12 for a, b in zip(r.energies, r.energies[1:]))
    assert r.energies[-1] < r.energies[0] - 1e-4
