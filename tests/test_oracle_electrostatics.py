"""Pins of the oracle's assembled electrostatics and of the reading on the ions' width.

1. The three electrostatic terms that the ground-state energy (Eq. GroundStateEnergy) adds
   together -- es = 1/2 int (u^2 + b) phi, the self-energy term -1/2 sum_J int b_J V_J and the
   overlap correction E_c^* (App. B) -- are checked as a sum, not one by one.  For a uniform
   electron density rho_bar = N_e / Omega and Gaussian ions of width sigma, their sum is the
   energy of point ions in a neutralising background (an Ewald sum, written here
   independently of the oracle and itself pinned by the published Madelung constant of the
   FCC lattice) plus the term the ions' width adds, 2 pi sigma^2 N_e^2 / Omega:
     * 1/2 int (rho_bar + b) phi is the energy of Gaussian ions in the background: the point-ion
       energy, plus each Gaussian's self energy Z^2 / (2 sqrt(pi) sigma), minus the erfc part
       of every pair (the overlap of two Gaussians, Z_I Z_J erfc(R / 2 sigma) / R), plus each
       ion's changed interaction with the background, rho_bar Z 4 pi int r erfc(r / (sqrt 2
       sigma)) dr = 2 pi rho_bar Z sigma^2;
     * the self-energy term removes the first, E_c^* adds back the second.
   A sign slip or a wrong factor on any of the three terms breaks the sum; the test goes
   through ground_state_energy itself, with the uniform-gas closed forms for TF and LDA.
2. Reading R6 (Gaussian width 1.2 bohr, not 0.7, for the cells run with the kernel term): along
   the energy's first descent direction from the uniform density, the full WT-type energy of
   the 4-atom cell with sigma = 0.7 ions is still falling where the density first reaches zero,
   while with sigma = 1.2 it has an interior minimum with u > 0.
"""
from math import pi, sqrt

import numpy as np
from scipy.special import erfc

import oracle as O
from oracle.scf import inner
from paper_1412_8250_gb300 import workloads as W

# Madelung energy of the FCC lattice of point charges Z in a uniform neutralising background,
# per ion: -0.895873615195 Z^2 / r_ws, r_ws the Wigner-Seitz radius (the standard value for
# the fcc lattice, e.g. the table of lattice Madelung constants of one-component plasmas)
FCC_MADELUNG_WS = 0.895873615195


def ewald_energy(R, Z, L, eta=0.6, nsig=7.0):
    """Energy of point charges Z_i at R_i (orthorhombic cell L, periodic) in a uniform
    neutralising background: real-space erfc sum, reciprocal-space sum, the point-charge self
    term and the background term -pi Q^2 / (2 Omega eta^2)."""
    R, Z, L = np.asarray(R, float), np.asarray(Z, float), np.asarray(L, float)
    omega, Q = float(np.prod(L)), float(Z.sum())
    rcut, gcut = nsig / eta, 2.0 * eta * nsig
    e_real = 0.0
    nmax = [int(np.ceil(rcut / L[d])) + 1 for d in range(3)]
    for a in range(-nmax[0], nmax[0] + 1):
        for b in range(-nmax[1], nmax[1] + 1):
            for c in range(-nmax[2], nmax[2] + 1):
                T = np.array([a, b, c]) * L
                d = np.linalg.norm(R[:, None, :] - R[None, :, :] - T, axis=2)
                if a == 0 and b == 0 and c == 0:
                    np.fill_diagonal(d, np.inf)
                m = d < rcut
                e_real += 0.5 * float(np.sum((Z[:, None] * Z[None, :] * erfc(eta * d) / d)[m]))
    e_rec = 0.0
    mmax = [int(np.ceil(gcut * L[d] / (2 * pi))) for d in range(3)]
    for a in range(-mmax[0], mmax[0] + 1):
        for b in range(-mmax[1], mmax[1] + 1):
            for c in range(-mmax[2], mmax[2] + 1):
                if a == b == c == 0:
                    continue
                G = 2 * pi * np.array([a, b, c]) / L
                G2 = float(G @ G)
                if G2 > gcut**2:
                    continue
                S = np.sum(Z * np.exp(1j * (R @ G)))
                e_rec += 2 * pi / omega * np.exp(-G2 / (4 * eta**2)) / G2 * abs(S) ** 2
    return e_real + e_rec - eta / sqrt(pi) * float(np.sum(Z**2)) - pi * Q**2 / (2 * omega * eta**2)


def test_ewald_sum_reproduces_the_fcc_madelung_energy():
    cell = W.al4_cell()
    rws = (3.0 * cell.L[0] ** 3 / (4.0 * pi * 4)) ** (1.0 / 3.0)
    ref = -FCC_MADELUNG_WS * 9.0 / rws * 4
    for eta in (0.4, 0.6, 0.9):   # the split parameter must not matter
        assert abs(ewald_energy(cell.R, cell.Z, cell.L, eta=eta) - ref) < 1e-9


def _uniform_energy(cell, n):
    grid = O.Grid((n, n, n), cell.L, 6)
    Ne = float(np.sum(cell.Z))
    rho = Ne / grid.volume
    u = np.full(grid.shape, sqrt(rho))
    b = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    phi = O.poisson_solve(u * u + b, grid)
    E, t = O.ground_state_energy(u, phi, b, grid, O.tfw_functional(), 0.0,
                                 O.self_energy(cell.R, cell.Z, cell.sigma, cell.rc, grid),
                                 O.repulsive_correction(cell.R, cell.Z, cell.sigma, grid.L))
    return E, t, grid, rho


def test_assembled_electrostatics_equal_the_ewald_energy_plus_the_width_term():
    cases = [(W.al4_lr_cell(), 32, 1e-9),                          # displaced, sigma = 1.2
             (W.fcc_supercell((1, 1, 1), sigma=1.2, rc=10.0), 32, 1e-9),
             (W.al4_cell(), 32, 1e-7)]                              # sigma = 0.7, h^12 error
    for cell, n, tol in cases:
        E, t, grid, rho = _uniform_energy(cell, n)
        Ne = float(np.sum(cell.Z))
        width = 2.0 * pi * cell.sigma**2 * Ne**2 / grid.volume
        ref_es = ewald_energy(cell.R, cell.Z, cell.L) + width
        tf = O.C_F * rho ** (5.0 / 3.0) * grid.volume
        xc = grid.volume * rho * float(O.eps_xc(np.array(rho)))
        assert abs(t["vw"]) < 1e-12
        assert abs(t["es"] + t["self"] + t["corr"] - ref_es) < tol, (cell.name, t)
        assert abs(E - (tf + xc + ref_es)) < tol, cell.name
        # the overlap term is large enough at sigma = 1.2 for a wrong factor to show
        if cell.sigma == 1.2:
            assert t["corr"] > 1e3 * tol


def _line_scan(sigma, rc, n_points=41):
    """Full WT-type energy along u(s) = sqrt(N_e) (u0 + s r) / ||u0 + s r|| from the uniform
    density u0, r = -2 (H u0 - eta u0) its constrained steepest-descent direction, for s from 0
    to just before the first point where u reaches zero."""
    cell = W.fcc_supercell((1, 1, 1), points_per_cell=16, displacement=0.1, seed=2, sigma=sigma,
                           rc=rc)
    grid = O.Grid(cell.n, cell.L, 6)
    Ne = float(np.sum(cell.Z))
    fn = O.wt_functional()
    kf2 = O.kf2_of(Ne, grid.volume)
    b = O.pseudocharge(cell.R, cell.Z, sigma, rc, grid)
    e_self = O.self_energy(cell.R, cell.Z, sigma, rc, grid)
    e_c = O.repulsive_correction(cell.R, cell.Z, sigma, grid.L)

    def energy(u):
        phi = O.poisson_solve(u * u + b, grid)
        V, T, _, _ = O.lr_potential(u, grid, fn, kf2)
        return O.ground_state_energy(u, phi, b, grid, fn, T, e_self, e_c)[0], phi, V

    u0 = np.full(grid.shape, sqrt(Ne / grid.volume))
    _, phi0, V0 = energy(u0)
    Hu = O.hamiltonian_apply(u0, phi0, V0, grid, fn)
    r = -2.0 * (Hu - inner(u0, Hu, grid) / Ne * u0)
    s_zero = u0.flat[0] / float(np.max(-r))          # u0 + s r first reaches zero here
    Es, umin = [], []
    for s in np.linspace(0.0, 0.999 * s_zero, n_points):
        w = u0 + s * r
        u = sqrt(Ne / inner(w, w, grid)) * w
        Es.append(energy(u)[0])
        umin.append(float(u.min()))
    return np.array(Es), np.array(umin)


def test_hard_ions_leave_the_kernel_functional_without_a_minimiser_on_the_descent_line():
    E07, u07 = _line_scan(0.7, 7.0)
    assert np.all(u07 > 0)
    assert np.all(np.diff(E07) < 0)                 # falling all the way to u = 0
    E12, u12 = _line_scan(1.2, 10.0)
    assert np.all(u12 > 0)
    k = int(np.argmin(E12))
    assert 0 < k < len(E12) - 1                     # an interior minimum with u > 0
    assert E12[-1] - E12[k] > 0.1
