"""Pins of the oracle's grid-evaluated overlap correction E_c^* with reference charges (App. B,
Eq. RepulsiveCorrection2 and the force expression after it)."""
import numpy as np

import oracle as O
from oracle.overlap import (repulsive_correction_grid, repulsive_correction_grid_forces,
                            repulsive_correction_pairs)
from paper_1412_8250_gb300 import workloads as W

SIGMA, RC = 1.2, 10.0           # overlapping ion charges (nearest neighbours 5.37 bohr apart)
SIGMA_REF, RC_REF = 0.5, 4.5    # reference charges that do not overlap


def _cell():
    return W.fcc_supercell((1, 1, 1), points_per_cell=32, displacement=0.15, seed=11,
                           sigma=SIGMA, rc=RC)


def test_reference_equal_to_the_charge_gives_no_correction():
    cell = _cell()
    grid = O.Grid((16, 16, 16), cell.L, 6)
    E, Vc, _ = repulsive_correction_grid(cell.R, cell.Z, SIGMA, RC, SIGMA, RC, grid)
    assert E == 0.0 and np.abs(Vc).max() == 0.0
    F = repulsive_correction_grid_forces(cell.R, cell.Z, SIGMA, RC, SIGMA, RC, grid, cutoff=6.0)
    assert np.abs(F).max() == 0.0


def test_energy_converges_to_the_pair_sum_at_order_2n():
    # the grid route (reference charges sampled, one periodic Poisson solve, self integrals
    # by quadrature) against the real-space pair sum of erfc terms, which shares nothing with
    # it; measured: errors 6.8e-5, 6.3e-6, 8.4e-7 Ha at 32, 40, 48 points per 7.6 bohr (order
    # ~11 for the order-12 stencil on the narrow reference charges)
    cell = _cell()
    ref = repulsive_correction_pairs(cell.R, cell.Z, SIGMA, SIGMA_REF, cell.L)
    # the reference charges do not overlap: the pair sum equals the point-reference closed form
    assert abs(ref - O.repulsive_correction(cell.R, cell.Z, SIGMA, cell.L)) < 1e-11
    errs = []
    ns = (32, 40, 48)
    for n in ns:
        grid = O.Grid((n, n, n), cell.L, 6)
        errs.append(abs(repulsive_correction_grid(cell.R, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF,
                                                  grid)[0] - ref))
    order = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert min(order) > 9.0, (errs, order)
    assert errs[-1] < 2e-6


def test_forces_match_the_pair_sum_and_the_grid_energy():
    cell = _cell()
    grid = O.Grid((24, 24, 24), cell.L, 6)
    F = repulsive_correction_grid_forces(cell.R, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF, grid)
    # the derivative of the pair sum (the reference term erfc(R / 2 sigma_ref) is below 1e-13
    # at these distances); the grid energy's error does not depend on the positions
    Fp = O.repulsive_correction_forces(cell.R, cell.Z, SIGMA, cell.L)
    assert np.abs(F - Fp).max() < 1e-9
    assert np.abs(F.sum(axis=0)).max() < 1e-10
    # central differences of the grid energy itself
    d = 1e-4
    for J, c in ((1, 0), (2, 2), (3, 1)):
        Rp, Rm = cell.R.copy(), cell.R.copy()
        Rp[J, c] += d
        Rm[J, c] -= d
        Ep = repulsive_correction_grid(Rp, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF, grid)[0]
        Em = repulsive_correction_grid(Rm, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF, grid)[0]
        assert abs(-(Ep - Em) / (2 * d) - F[J, c]) < 1e-8, (J, c)
