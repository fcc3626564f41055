"""Writes tests/golden/ground_states.json: oracle ground states of two small cells.

Calls only the oracle (and the seeded input generator for the ion positions, which are
stored alongside the results so every consumer reads identical inputs).
  al4_tfw : 4-atom FCC cell, a = 7.6, 32^3, 12th-order FD, TFW (lambda = 1/5) + PZ LDA,
            Gaussian ions Z = 3, sigma = 0.7, r_c = 7, uniform initial density.
  al4_wt  : 4-atom FCC cell with +-0.1 displacements (seed 2), 32^3, WT-type kernel term,
            Gaussian ions Z = 3, sigma = 1.2, r_c = 10, Anderson m = 7, zeta = 0.3.
Usage: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import workloads as W  # noqa: E402


def run(cell, fn, name, **kw):
    grid = O.Grid(cell.n, cell.L, 6)
    t = time.time()
    res = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, fn, **kw)
    F = O.forces(res.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    return dict(name=name, n=list(cell.n), L=list(cell.L), R=cell.R.tolist(), Z=cell.Z.tolist(),
                sigma=cell.sigma, rc=cell.rc, fd_half_order=6, energy=res.energy,
                terms={k: float(v) for k, v in res.terms.items()},
                energy_per_atom=res.energy / cell.n_atoms, forces=F.tolist(),
                nlcg_iterations=res.nlcg_iterations, fp_errors=res.fp_errors,
                options={k: v for k, v in kw.items()}, seconds=time.time() - t)


if __name__ == "__main__":
    out = {}
    out["al4_tfw"] = run(W.al4_cell(), O.tfw_functional(), "al4_tfw", nlcg_tol=1e-7)
    out["al4_wt"] = run(W.al4_lr_cell(), O.wt_functional(), "al4_wt", nlcg_tol=1e-7,
                        fp_tol=1e-7, anderson_m=7, zeta=0.3)
    with open(os.path.join(HERE, "ground_states.json"), "w") as f:
        json.dump(out, f, indent=1)
    for k, v in out.items():
        print(k, v["energy"], v["nlcg_iterations"], v["seconds"])
