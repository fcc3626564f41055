"""Plain FP64 CPU oracle for the periodic orbital-free DFT hot path.

Ghosh & Suryanarayana, "Higher-order finite-difference formulation of periodic Orbital-free
Density Functional Theory" (arXiv:1412.8250).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference leg, and by
nothing else.  The CUDA product path never imports it, and it imports nothing from the
product package: the two share no code.  Inputs come from the seeded generators in
``paper_1412_8250_gb300.workloads`` (passed in by the caller as plain numpy arrays).

Everything here is slow on purpose: numpy, float64, no blocking, no fusion, each function
citing the passage of the paper it restates.  Fields are numpy arrays of shape
(n3, n2, n1), x fastest.

Parity status per function is listed in each module's header; every function is pinned by
``tests/test_oracle_*.py`` against closed forms, brute force, invariants or finite
differences (none is "parity unpinned").
"""
from .fd import Grid, fd_laplacian_weights, fd_gradient_weights, laplacian, gradient, integrate
from .fd import laplacian_symbol, solve_shifted_spectral, poisson_solve
from .pseudo import (pseudocharge, self_energy, repulsive_correction,
                     repulsive_correction_forces, gaussian_b, gaussian_V, atom_box)
from .functional import (C_F, tf_energy_density, tf_potential, xc_energy_density,
                         eps_xc, v_xc, PZ)
from .kernel import (WGC_TABLE, wt_functional, wgc_functional, Functional, tfw_functional,
                     kernel_solve, lr_potential, lr_potential_wgc, kernel_class, c_mnpq,
                     rho_bar_of, kf2_of)
from .scf import (hamiltonian_apply, inner_energy, nlcg, anderson_update, scf_ground_state,
                  ground_state_energy, ScfResult)
from .forces import forces
from .relax import relax, RelaxResult
from .vacancy import vacancy_cell, vacancy_formation, VacancyResult
from .overlap import (repulsive_correction_grid, repulsive_correction_grid_forces,
                      repulsive_correction_pairs)

__all__ = [n for n in dir() if not n.startswith("_")]
