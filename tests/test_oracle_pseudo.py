"""Pins of the oracle's pseudocharges, self energy and overlap correction (Sec. 3.2, App. B)."""
from math import pi, sqrt

import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W


@pytest.mark.parametrize("cell", [W.al4_cell(), W.al4_lr_cell(), W.fcc_supercell((2, 1, 1), displacement=0.1, seed=1)])
def test_neutrality(cell):
    grid = O.Grid(cell.n, cell.L, 6)
    b = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    assert abs(grid.dV * b.sum() + cell.Z.sum()) < 1e-10 * cell.Z.sum()
    assert b.max() <= 0.0


def test_pseudocharge_is_minus_laplacian_of_potential():
    # b_J = -(1/4 pi) lap V_J in the continuum (Eq. b:Pseudopotential): check with a fine
    # radial finite difference of r V(r) at several radii
    Z, s = 3.0, 0.7
    for r in [0.3, 0.9, 1.7, 3.0]:
        e = 1e-3
        rv = lambda x: x * O.gaussian_V(np.array([x]), Z, s)[0]
        lap = (rv(r + e) - 2 * rv(r) + rv(r - e)) / (e * e) / r
        assert abs(-lap / (4 * pi) - O.gaussian_b(r, Z, s)) < 1e-6 * abs(O.gaussian_b(0.0, Z, s))


def test_self_energy_continuum_value():
    c = W.al4_cell()
    grid = O.Grid(c.n, c.L, 6)
    e = O.self_energy(c.R, c.Z, c.sigma, c.rc, grid)
    ref = -0.5 * np.sum(c.Z**2) / (sqrt(pi) * c.sigma)
    assert abs(e - ref) < 1e-9 * abs(ref)


def test_gaussian_pair_interaction_matches_erf_form():
    # int b_I V_J for two isolated Gaussians equals Z^2 erf(R/(2 sigma))/R -- the identity
    # behind E_c^*; quadrature on a fine grid around ion I
    Z, s, R = 3.0, 0.7, 1.9
    h = 0.05
    ax = np.arange(-5.0, 5.0 + h / 2, h)
    x, y, z = np.meshgrid(ax, ax, ax, indexing="ij")
    rI = np.sqrt(x**2 + y**2 + z**2)
    rJ = np.sqrt((x - R) ** 2 + y**2 + z**2)
    val = h**3 * np.sum(O.gaussian_b(rI, Z, s) * O.gaussian_V(rJ, Z, s))
    from scipy.special import erf
    assert abs(val - Z * Z * erf(R / (2 * s)) / R) < 1e-6


def test_repulsive_correction_isolated_pairs_against_quadrature():
    # A large cell with three close ions: only T = 0 pairs are within the cutoff, so
    # E_c^* = sum_{I<J} [Z^2/R_IJ - int b_I V_J]; the integral by direct quadrature.
    Z, s = 3.0, 0.7
    R = np.array([[20.0, 20.0, 20.0], [21.3, 20.4, 20.0], [20.2, 21.5, 19.1]])
    Zs = np.full(3, Z)
    e = O.repulsive_correction(R, Zs, s, (40.0, 40.0, 40.0))
    h = 0.05
    ax = np.arange(-5.0, 5.0 + h / 2, h)
    x, y, z = np.meshgrid(ax, ax, ax, indexing="ij")
    ref = 0.0
    for I in range(3):
        for J in range(I + 1, 3):
            d = R[J] - R[I]
            rI = np.sqrt(x**2 + y**2 + z**2)
            rJ = np.sqrt((x - d[0]) ** 2 + (y - d[1]) ** 2 + (z - d[2]) ** 2)
            inter = h**3 * np.sum(O.gaussian_b(rI, Z, s) * O.gaussian_V(rJ, Z, s))
            ref += Z * Z / np.linalg.norm(d) - inter
    assert abs(e - ref) < 1e-6 * abs(ref)


def test_repulsive_correction_is_extensive():
    # E_c^* of a 2x2x2 replica equals 8x the cell's (catches missing periodic images)
    c = W.fcc_supercell((1, 1, 1), displacement=0.3, seed=4, sigma=1.2)
    e1 = O.repulsive_correction(c.R, c.Z, c.sigma, c.L)
    R8 = np.concatenate([c.R + np.array([i, j, k]) * 7.6 for i in range(2) for j in range(2) for k in range(2)])
    e8 = O.repulsive_correction(R8, np.full(len(R8), 3.0), c.sigma, (15.2, 15.2, 15.2))
    assert abs(e8 - 8 * e1) < 1e-10 * abs(e8)
    assert e1 > 0


def test_repulsive_correction_forces_finite_difference():
    c = W.fcc_supercell((1, 1, 1), displacement=0.4, seed=5, sigma=1.2)
    F = O.repulsive_correction_forces(c.R, c.Z, c.sigma, c.L)
    d = 1e-5
    for J in [0, 2]:
        for a in range(3):
            Rp, Rm = c.R.copy(), c.R.copy()
            Rp[J, a] += d
            Rm[J, a] -= d
            fd = -(O.repulsive_correction(Rp, c.Z, c.sigma, c.L) - O.repulsive_correction(Rm, c.Z, c.sigma, c.L)) / (2 * d)
            assert abs(fd - F[J, a]) < 1e-7 + 1e-5 * abs(F[J, a])
    assert np.max(np.abs(F.sum(0))) < 1e-10


def test_pseudocharge_from_the_potential_converges_to_the_gaussian():
    # b_J = -(1/4pi) L_h V_J (the paper's construction from the potential, Sec. 4) against the
    # closed-form Gaussian charge it discretises: the gap closes at the order of the scheme,
    # the ions stay neutral, and the self energy converges with it
    from oracle.pseudo import pseudocharge_fd
    errs = []
    for ppc in (24, 32):
        cell = W.al4_cell(points_per_cell=ppc)
        g = O.Grid(cell.n, cell.L, 6)
        bfd, es_fd = pseudocharge_fd(cell.R, cell.Z, cell.sigma, cell.rc, g)
        ba = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, g)
        errs.append(np.abs(bfd - ba).max() / np.abs(ba).max())
        assert abs(bfd.sum() * g.dV + cell.Z.sum()) <= 1e-9 * cell.Z.sum()
        es = O.self_energy(cell.R, cell.Z, cell.sigma, cell.rc, g)
        assert abs(es_fd - es) <= 1e-4 * abs(es)
    assert errs[1] < 1e-6 and errs[1] < errs[0] * (24 / 32) ** 8, errs
