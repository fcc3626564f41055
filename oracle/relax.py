"""Geometry relaxation (Sec. 3.3, last paragraph of "Determining the ground state": the
equilibrium positions of the nuclei by non-linear conjugate gradients with the Polak-Ribiere
update and a secant line search, Shewchuk's formulation).

Oracle (test infrastructure only).  Each force evaluation is a full ground state
(scf_ground_state, warm-started from the density of the previous evaluation) followed by
forces().

Readings (the paper names the method only):
  * objective E(R), gradient -F(R); the search direction starts along F, then
    d = F_k + beta d_{k-1} with beta = max(0, F_k . (F_k - F_{k-1}) / F_{k-1} . F_{k-1})
    (Polak-Ribiere with the usual restart at beta < 0), and restarts along F whenever d is not
    a descent direction;
  * the line search finds the root of E'(s) = -F(R + s d) . d by the secant method, from
    E'(0) (the current forces) and a trial step that moves the farthest atom by `step0` bohr;
    it stops when |E'(s)| <= line_tol |E'(0)| or after max_line secant points, and the last
    point is accepted (its ground state and forces start the next step);
  * convergence: max_J |F_J| < ftol.

Pins (tests/test_oracle_relax.py): one atom displaced from a perfect FCC cell relaxes back to
the perfect lattice (up to the common translation the forces cannot see); the energy of every
accepted step is below the starting energy; the final forces are below ftol.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .fd import Grid
from .forces import forces
from .kernel import Functional
from .scf import scf_ground_state


@dataclass
class RelaxResult:
    R: np.ndarray
    energy: float
    max_force: float
    steps: int
    evaluations: int
    energies: list = field(default_factory=list)
    u: np.ndarray | None = None


def relax(grid: Grid, R0, Z, sigma, rc, fn: Functional, ftol=1e-3, max_steps=40, step0=0.05,
          line_tol=0.1, max_line=4, **scf_kw) -> RelaxResult:
    R = np.array(R0, dtype=float)
    Z = np.asarray(Z, dtype=float)

    def evaluate(Rx, u0):
        res = scf_ground_state(grid, Rx, Z, sigma, rc, fn, u0=u0, **scf_kw)
        return res, forces(res.phi, Rx, Z, sigma, rc, grid)

    res, F = evaluate(R, None)
    evals = 1
    energies = [res.energy]
    d = F.copy()
    F_prev = None
    steps = 0
    while steps < max_steps and np.abs(F).max() >= ftol:
        if F_prev is not None:
            beta = max(0.0, float(np.sum(F * (F - F_prev)) / np.sum(F_prev * F_prev)))
            d = F + beta * d
        g0 = -float(np.sum(F * d))            # E'(0) along d
        if not g0 < 0.0:                      # not a descent direction: restart along F
            d = F.copy()
            g0 = -float(np.sum(F * F))
        s_a, g_a = 0.0, g0
        s = step0 / np.abs(d).max()
        u_warm = res.u
        for j in range(max_line):
            res_s, F_s = evaluate(R + s * d, u_warm)
            u_warm = res_s.u
            evals += 1
            g = -float(np.sum(F_s * d))
            if abs(g) <= line_tol * abs(g0) or j + 1 == max_line:
                break
            if g > g_a:                       # secant root of E'(s) through the last two points
                s_new = s - g * (s - s_a) / (g - g_a)
            else:                             # no positive curvature seen: step further
                s_new = 2.0 * s
            s_a, g_a = s, g
            s = s_new
        F_prev = F
        R = R + s * d
        res, F = res_s, F_s
        energies.append(res.energy)
        steps += 1
    return RelaxResult(R=R, energy=res.energy, max_force=float(np.abs(F).max()), steps=steps,
                       evaluations=evals, energies=energies, u=res.u)
