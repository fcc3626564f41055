"""Vacancy formation energy (Sec. 5.6, "Vacancy formation energy in Aluminum").

Oracle (test infrastructure only).  The formation energy of one vacancy follows the relation
the paper uses, with E(M, n, Omega) the energy of a periodic cell of volume Omega with M occupied
lattice sites and n vacancies:

    E_vf = E(M - 1, 1, (M - 1)/M Omega) - ((M - 1)/M) E(M, 0, Omega).

The vacancy cell keeps the volume per atom of the perfect cell: every length (cell sides and
the remaining positions) is scaled by s = ((M - 1)/M)^{1/3} about the origin, on a grid with the
same number of points (so h shrinks by s as well).  The unrelaxed value takes the scaled lattice
sites; the relaxed one relaxes the vacancy cell's ions (relax.py) at that fixed volume.

Readings (the paper states the relation only):
  * the perfect cell's lattice constant is the caller's (the paper's is the stress-free one;
    finding it is the bulk-modulus workflow, not built);
  * the removed site is the caller's index into the perfect cell's ions;
  * the vacancy cell's ground state starts from the uniform density, its relaxation from the
    unrelaxed ground state.

Pins (tests/test_oracle_vacancy.py): the vacancy cell's volume is (M - 1)/M of the perfect one
and its electron count Ne - Z_site; removing any of the sites of a perfect FCC cell gives the
same E_vf (the sites are related by lattice translations that map the grid onto itself); the
relaxed E_vf is at most the unrelaxed one and equals it when the remaining ions sit on
inversion centres (the 4-atom cell).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .fd import Grid
from .kernel import Functional
from .relax import relax
from .scf import scf_ground_state


@dataclass
class VacancyResult:
    e_perfect: float
    e_unrelaxed: float
    e_relaxed: float
    evf_unrelaxed: float
    evf_relaxed: float
    R_vacancy: np.ndarray      # final positions of the vacancy cell's ions
    grid_vacancy: Grid
    relax_steps: int = 0
    evaluations: int = 0
    max_force: float = 0.0


def vacancy_cell(grid: Grid, R, Z, site: int):
    """The vacancy cell of a perfect cell (grid, R, Z): site removed, lengths scaled by
    ((M - 1)/M)^{1/3}, same grid point counts."""
    R = np.asarray(R, dtype=float)
    Z = np.asarray(Z, dtype=float)
    M = R.shape[0]
    if not 0 <= site < M or M < 2:
        raise ValueError("site out of range")
    s = ((M - 1) / M) ** (1.0 / 3.0)
    vgrid = Grid(grid.n, tuple(s * L for L in grid.L), grid.N)
    Rv = s * np.delete(R, site, axis=0)
    Zv = np.delete(Z, site)
    return vgrid, Rv, Zv


def vacancy_formation(grid: Grid, R, Z, sigma, rc, fn: Functional, site: int, relaxed=False,
                      relax_kw=None, **scf_kw) -> VacancyResult:
    M = np.asarray(R).shape[0]
    perfect = scf_ground_state(grid, R, Z, sigma, rc, fn, **scf_kw)
    vgrid, Rv, Zv = vacancy_cell(grid, R, Z, site)
    frac = (M - 1) / M
    if relaxed:
        r = relax(vgrid, Rv, Zv, sigma, rc, fn, **(relax_kw or {}), **scf_kw)
        e_unrel, e_rel = r.energies[0], r.energy
        out = dict(R_vacancy=r.R, relax_steps=r.steps, evaluations=r.evaluations,
                   max_force=r.max_force)
    else:
        e_unrel = scf_ground_state(vgrid, Rv, Zv, sigma, rc, fn, **scf_kw).energy
        e_rel = e_unrel
        out = dict(R_vacancy=Rv)
    return VacancyResult(e_perfect=perfect.energy, e_unrelaxed=e_unrel, e_relaxed=e_rel,
                         evf_unrelaxed=e_unrel - frac * perfect.energy,
                         evf_relaxed=e_rel - frac * perfect.energy, grid_vacancy=vgrid, **out)
