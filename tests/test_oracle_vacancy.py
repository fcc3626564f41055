"""Pins of the oracle's vacancy formation energy (Sec. 5.6: E_vf = E(M-1, 1, (M-1)/M Omega)
- ((M-1)/M) E(M, 0, Omega))."""
import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W


def test_vacancy_cell_keeps_the_volume_per_atom():
    cell = W.fcc_supercell((2, 1, 1), points_per_cell=12, displacement=0.1, seed=7)
    grid = O.Grid(cell.n, cell.L, 6)
    M = cell.n_atoms
    for site in (0, 3, M - 1):
        vg, Rv, Zv = O.vacancy_cell(grid, cell.R, cell.Z, site)
        assert vg.n == grid.n and vg.N == grid.N
        assert abs(vg.volume - (M - 1) / M * grid.volume) <= 1e-13 * grid.volume
        assert abs(vg.volume / Rv.shape[0] - grid.volume / M) <= 1e-13 * grid.volume / M
        assert Zv.sum() == cell.Z.sum() - cell.Z[site] and Rv.shape == (M - 1, 3)
        # the remaining ions keep their fractional coordinates
        keep = np.delete(np.arange(M), site)
        frac_v = Rv / np.array(vg.L)
        frac_p = cell.R[keep] / np.array(grid.L)
        assert np.abs(frac_v - frac_p).max() <= 1e-14
    with pytest.raises(ValueError):
        O.vacancy_cell(grid, cell.R, cell.Z, M)


def test_every_site_of_a_perfect_cell_gives_the_same_formation_energy():
    # the FCC sites are related by lattice translations of a/2 that map the grid (12 points
    # per cell edge) onto itself, so the vacancy cells are translates of one another and the
    # energies agree to rounding: a wrong site removed, a position left unscaled or a scaling
    # about another origin breaks it
    cell = W.al4_cell(points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    fn = O.tfw_functional()
    evf = [O.vacancy_formation(grid, cell.R, cell.Z, cell.sigma, cell.rc, fn, s,
                               nlcg_tol=1e-9).evf_unrelaxed for s in range(4)]
    assert all(abs(e - evf[0]) <= 1e-11 for e in evf), evf
    # a positive formation energy of a few tenths of an eV for this Al-like cell
    assert 0.005 < evf[0] < 0.05


def test_relaxation_lowers_the_formation_energy():
    fn = O.tfw_functional()
    # 4-atom cell: the three remaining ions sit on inversion centres, no force, no step
    cell = W.al4_cell(points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    r = O.vacancy_formation(grid, cell.R, cell.Z, cell.sigma, cell.rc, fn, 0, relaxed=True,
                            relax_kw=dict(ftol=1e-5), nlcg_tol=1e-9)
    assert r.relax_steps == 0 and r.max_force < 1e-10
    assert r.evf_relaxed == r.evf_unrelaxed
    # 8-atom cell: the neighbours of the vacancy move and the energy drops
    cell = W.fcc_supercell((2, 1, 1), points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    r = O.vacancy_formation(grid, cell.R, cell.Z, cell.sigma, cell.rc, fn, 0, relaxed=True,
                            relax_kw=dict(ftol=1e-4), nlcg_tol=1e-9)
    assert r.relax_steps >= 1 and r.max_force < 1e-4
    assert r.evf_relaxed < r.evf_unrelaxed - 5e-4
    # the relaxed ions keep the cell's mirror symmetry through the vacancy (x -> -x about the
    # removed site at the origin maps the remaining sites onto themselves)
    Rv0 = O.vacancy_cell(grid, cell.R, cell.Z, 0)[1]
    Lv = np.array(r.grid_vacancy.L)
    disp = r.R_vacancy - Rv0
    mirror = np.mod(-Rv0[:, 0], Lv[0])
    for i in range(Rv0.shape[0]):
        j = int(np.argmin(np.abs(np.mod(Rv0[:, 0] - mirror[i] + Lv[0] / 2, Lv[0]) - Lv[0] / 2)
                          + np.abs(Rv0[:, 1] - Rv0[i, 1]) + np.abs(Rv0[:, 2] - Rv0[i, 2])))
        assert abs(disp[i, 0] + disp[j, 0]) < 2e-3 and abs(disp[i, 1] - disp[j, 1]) < 2e-3
