"""Writes the oracle's stored ground states under tests/golden/.

Calls only the oracle (and the seeded input generator for the ion positions, which are
stored alongside the results so every consumer reads identical inputs).

ground_states.json (the default):
  al4_tfw : 4-atom FCC cell, a = 7.6, 32^3, 12th-order FD, TFW (lambda = 1/5) + PZ LDA,
            Gaussian ions Z = 3, sigma = 0.7, r_c = 7, uniform initial density.
  al4_wt  : 4-atom FCC cell with +-0.1 displacements (seed 2), 32^3, WT-type kernel term,
            Gaussian ions Z = 3, sigma = 1.2, r_c = 10, Anderson m = 7, zeta = 0.3.
al108_wt.json (--al108; about half an hour on one host core):
  al108_wt: 108-atom 3x3x3 FCC cell with +-0.1 displacements (seed 2), 96^3, 12th-order FD,
            WT-type kernel term, sigma = 1.2, r_c = 10, Anderson m = 3, zeta = 1 (the paper's
            choice for linear-response runs, Sec. 5.3), every inner solve exact, fixed point
            to 1e-7.  Besides the energy, its terms and the forces, the record keeps the NLCG
            steps of every outer iteration and the number of outer iterations (one kernel map
            each), from which a per-ground-state oracle time can be rebuilt from a timed
            sample, and the oracle's own wall time for the whole ground state.
batched_cells.json (--batched; two processes, each about 15 to 25 minutes on one host core):
  the two smallest cells of the 64-cell set (W.batched_cells(), seed 3): cell15, 2x2x2 FCC,
  32 atoms, 64^3, and cell11, 2x2x3 FCC with one site removed, 47 atoms, 64 x 64 x 96; +-0.1
  bohr displacements, WT-type kernel term, sigma = 1.2, r_c = 10, Anderson m = 3, zeta = 1,
  every inner solve exact, fixed point to 1e-7; the same record fields as al108_wt.
Usage: python tests/golden/make_golden.py [--al108 | --batched]
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
    t_gs = time.time() - t
    F = O.forces(res.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    return dict(name=name, n=list(cell.n), L=list(cell.L), R=cell.R.tolist(), Z=cell.Z.tolist(),
                sigma=cell.sigma, rc=cell.rc, fd_half_order=6, energy=res.energy,
                terms={k: float(v) for k, v in res.terms.items()},
                energy_per_atom=res.energy / cell.n_atoms, forces=F.tolist(),
                nlcg_iterations=res.nlcg_iterations, fp_errors=res.fp_errors,
                outer_iterations=res.outer_iterations,
                options={k: v for k, v in kw.items()}, seconds=time.time() - t,
                seconds_ground_state=t_gs)


BATCHED_GOLDEN = (15, 11)   # indices into W.batched_cells()


def run_batched_cell(index):
    cell = W.batched_cells()[index]
    return run(cell, O.wt_functional(), cell.name, nlcg_tol=1e-7, fp_tol=1e-7, anderson_m=3,
               zeta=1.0)


if __name__ == "__main__":
    if "--batched" in sys.argv:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(len(BATCHED_GOLDEN)) as pool:
            recs = pool.map(run_batched_cell, BATCHED_GOLDEN)
        with open(os.path.join(HERE, "batched_cells.json"), "w") as f:
            json.dump({r["name"]: r for r in recs}, f, indent=1)
        for r in recs:
            print(r["name"], r["energy"], r["nlcg_iterations"], r["seconds"])
        sys.exit(0)
    if "--al108" in sys.argv:
        rec = run(W.al108_cell(), O.wt_functional(), "al108_wt", nlcg_tol=1e-7, fp_tol=1e-7,
                  anderson_m=3, zeta=1.0)
        with open(os.path.join(HERE, "al108_wt.json"), "w") as f:
            json.dump({"al108_wt": rec}, f, indent=1)
        print("al108_wt", rec["energy"], rec["nlcg_iterations"], rec["seconds"])
        sys.exit(0)
    out = {}
    out["al4_tfw"] = run(W.al4_cell(), O.tfw_functional(), "al4_tfw", nlcg_tol=1e-7)
    out["al4_wt"] = run(W.al4_lr_cell(), O.wt_functional(), "al4_wt", nlcg_tol=1e-7,
                        fp_tol=1e-7, anderson_m=7, zeta=0.3)
    with open(os.path.join(HERE, "ground_states.json"), "w") as f:
        json.dump(out, f, indent=1)
    for k, v in out.items():
        print(k, v["energy"], v["nlcg_iterations"], v["seconds"])
