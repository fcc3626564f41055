"""The 64-cell set at full size: 64 independent FCC cells (2..4 repeats per axis, 64..128 points
per axis, 54.6 M points and 6,636 atoms in all, half with one site removed), WT-type kernel,
ground state + forces of every cell in one batched call with the benchmark's options.

Checked: every cell converges with the invariants of any size (constraint, positivity, a
mean-free phi, the momentum balance of its forces); the two smallest cells (cell15, 32 atoms,
64^3; cell11, 47 atoms with a vacancy, 64 x 64 x 96) against the oracle's own ground states
of those cells (tests/golden/batched_cells.json, written by tests/golden/make_golden.py
--batched from the oracle alone) at the 1e-6 Ha/atom and 1e-5 Ha/bohr bars; and the batched
result of those two and the largest cell equal, bit for bit, to a single-cell call.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
E_TOL = 1e-6   # Ha/atom
F_TOL = 1e-5   # Ha/bohr


@pytest.fixture(scope="module")
def batch():
    import bench
    cells = W.batched_cells()
    stream = torch.cuda.current_stream()
    _, h0, _, _, o = bench.make_case(torch, B, Fn, W, "mixed")
    B.of_grid_destroy(h0)
    fn = Fn.wt()
    grids = [B.of_grid_create(c.n, c.L, 6, stream) for c in cells]
    try:
        systems = [B.make_system(c.R, c.Z, c.sigma, c.rc) for c in cells]
        us = [torch.ones(c.shape, dtype=torch.float64, device="cuda") for c in cells]
        phis = [torch.zeros_like(x) for x in us]
        results = B.of_scf_ground_state_batched(grids, systems, fn, o, us, phis)
        forces = [B.of_forces(g, s, x, p) for g, s, x, p in zip(grids, systems, us, phis)]
        largest = int(np.argmax([c.n_points for c in cells]))
        single = {}
        for k in (15, 11, largest):
            u1 = torch.ones(cells[k].shape, dtype=torch.float64, device="cuda")
            p1 = torch.zeros_like(u1)
            r1 = B.of_scf_ground_state(grids[k], systems[k], fn, o, u1, p1)
            F1 = B.of_forces(grids[k], systems[k], u1, p1)
            single[k] = (r1, F1, torch.equal(u1, us[k]), torch.equal(p1, phis[k]))
        stats = []
        for c, x, p in zip(cells, us, phis):
            dV = float(np.prod(np.array(c.L) / np.array(c.n)))
            stats.append((float(torch.sum(x * x)) * dV, float(torch.min(x)),
                          float(torch.mean(p)), float(torch.max(torch.abs(p)))))
    finally:
        for g in grids:
            B.of_grid_destroy(g)
    return dict(cells=cells, results=results, forces=forces, single=single, stats=stats)


def test_every_cell_converges_with_its_invariants(batch):
    cells, results, forces, stats = batch["cells"], batch["results"], batch["forces"], batch["stats"]
    assert len(cells) == 64 and sum(c.n_points for c in cells) == 54624256
    assert sum(c.n_atoms for c in cells) == 6636
    for c, r, F, (ne, umin, pmean, pmax) in zip(cells, results, forces, stats):
        assert r.converged, c.name
        assert abs(ne - c.n_electrons) < 1e-9 * c.n_electrons, c.name
        assert umin > 0, c.name
        assert abs(pmean) < 1e-10 * pmax, c.name
        assert np.max(np.abs(F.sum(0))) < 1e-4, c.name


def test_smallest_cells_against_the_oracle(batch):
    with open(os.path.join(HERE, "golden", "batched_cells.json")) as f:
        gold = json.load(f)
    for k in (15, 11):
        c, r, F = batch["cells"][k], batch["results"][k], batch["forces"][k]
        rec = gold[c.name]
        assert np.array_equal(np.array(rec["R"]), c.R) and list(rec["n"]) == list(c.n)
        assert abs(r.energy - rec["energy"]) / c.n_atoms <= E_TOL, c.name
        assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL, c.name


def test_batched_equals_single_cell_calls(batch):
    for k, (r1, F1, u_same, phi_same) in batch["single"].items():
        r = batch["results"][k]
        assert r1.energy == r.energy, (k, r1.energy, r.energy)
        assert np.array_equal(F1, batch["forces"][k]), k
        assert u_same and phi_same, k
