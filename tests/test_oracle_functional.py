"""Pins of the oracle's Thomas-Fermi and Perdew-Zunger LDA terms (Sec. 2, Sec. 3.3.1)."""
from math import pi

import numpy as np
import pytest

import oracle as O


def test_cf_value():
    assert abs(O.C_F - 2.871234000188191) < 1e-12


def test_uniform_gas_closed_forms():
    rho, vol = 0.027336, 438.976
    grid = O.Grid((8, 8, 8), (vol ** (1 / 3),) * 3, 6)
    u = np.full(grid.shape, np.sqrt(rho))
    tf = O.integrate(O.tf_energy_density(u * u), grid)
    assert abs(tf - O.C_F * rho ** (5 / 3) * vol) < 1e-12 * tf
    vw = O.integrate(-0.5 * u * O.laplacian(u, grid), grid)
    assert abs(vw) < 1e-12
    ex = -0.75 * (3 / pi) ** (1 / 3) * rho ** (4 / 3) * vol
    rs = (3 / (4 * pi * rho)) ** (1 / 3)
    ec = -0.1423 / (1 + 1.0529 * np.sqrt(rs) + 0.3334 * rs) * rho * vol
    assert abs(O.integrate(O.xc_energy_density(u * u), grid) - (ex + ec)) < 1e-12 * abs(ex + ec)


@pytest.mark.parametrize("rho", [1e-4, 0.01, 0.027, 0.2, 0.5, 3.0])
def test_potentials_are_density_derivatives(rho):
    e = rho * 1e-5
    r = np.array([rho - e, rho + e])
    d_tf = (O.tf_energy_density(r[1]) - O.tf_energy_density(r[0])) / (2 * e)
    assert abs(d_tf - O.tf_potential(rho)) < 1e-8 * abs(d_tf)
    d_xc = (O.xc_energy_density(r[1]) - O.xc_energy_density(r[0])) / (2 * e)
    assert abs(d_xc - O.v_xc(np.array(rho))) < 1e-8 * abs(d_xc)


def test_pz_branch_split_and_continuity():
    rs1 = 3 / (4 * pi)           # rho at r_s = 1
    lo = O.eps_xc(np.array(rs1 * (1 + 1e-9)))  # r_s slightly below 1: log branch
    hi = O.eps_xc(np.array(rs1 * (1 - 1e-9)))
    assert abs(lo - hi) < 5e-5          # the printed constants make e_c continuous to ~3e-5
    assert abs(lo - hi) > 1e-7          # but the two branches are distinct formulas
