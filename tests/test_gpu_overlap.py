"""The overlap correction E_c^* and f^c evaluated on the grid with reference charges (App. B,
Eq. RepulsiveCorrection2; of_system.sigma_ref > 0) against the oracle's grid evaluation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle.overlap import repulsive_correction_grid, repulsive_correction_grid_forces  # noqa: E402
from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
SIGMA, RC, SIGMA_REF, RC_REF = 1.2, 10.0, 0.5, 4.5


def test_overlap_correction_on_the_grid_matches_oracle():
    # 4-atom cell with overlapping sigma = 1.2 ions, reference charges of width 0.5: the
    # energy term of a ground state and the force correction (of_forces with and without the
    # grid form, whose Hellmann-Feynman parts cancel) within 1e-9 of the oracle
    cell = W.fcc_supercell((1, 1, 1), points_per_cell=24, displacement=0.15, seed=11,
                           sigma=SIGMA, rc=RC)
    grid = O.Grid(cell.n, cell.L, 6)
    E_ref, _, _ = repulsive_correction_grid(cell.R, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF, grid)
    F_ref = repulsive_correction_grid_forces(cell.R, cell.Z, SIGMA, RC, SIGMA_REF, RC_REF, grid)
    Fc_closed = O.repulsive_correction_forces(cell.R, cell.Z, SIGMA, cell.L)
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        s_grid = B.make_system(cell.R, cell.Z, SIGMA, RC, sigma_ref=SIGMA_REF, rc_ref=RC_REF)
        s_closed = B.make_system(cell.R, cell.Z, SIGMA, RC)
        phi = torch.zeros(cell.shape, dtype=torch.float64, device="cuda")
        F_grid = B.of_forces(h, s_grid, phi, phi)
        F_closed = B.of_forces(h, s_closed, phi, phi)
        o = B.of_default_scf_opts()
        o.precision = B.OF_F32
        u = torch.ones_like(phi)
        res = B.of_scf_ground_state(h, s_grid, Fn.tfw(), o, u, phi)
    finally:
        B.of_grid_destroy(h)
    assert abs(res.e_corr - E_ref) < 1e-9
    # the Hellmann-Feynman part is the same in both calls: the difference is f^c alone
    assert np.abs((F_grid - F_closed) - (F_ref - Fc_closed)).max() < 1e-9
