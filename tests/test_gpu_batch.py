"""GPU parity of the batched Poisson solver against the oracle's exact discrete solutions, and
against the single-grid solver run cell by cell, in both forms: grouped launches over uneven
cells with one CUDA graph for the lockstep plain CG (no_multigrid), and the per-cell multigrid
solves spread over concurrent streams (the default)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import binding as B, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [((24, 24, 24), (5.7, 5.7, 5.7)), ((32, 16, 24), (7.6, 3.8, 5.7)),
          ((16, 16, 16), (3.8, 3.8, 3.8)), ((20, 28, 24), (4.75, 6.65, 5.7)),
          ((48, 40, 32), (11.4, 9.5, 7.6)), ((12, 12, 36), (2.85, 2.85, 8.55))]


def _opts(tol, multigrid=True):
    o = B.of_default_solve_opts()
    o.tol = tol
    o.precision = B.OF_F32
    o.no_multigrid = 0 if multigrid else 1
    return o


@pytest.mark.parametrize("multigrid", [False, True], ids=["grouped_cg", "concurrent_multigrid"])
def test_batched_poisson_matches_oracle_and_single_grid(multigrid):
    stream = torch.cuda.current_stream()
    grids, rhos, phis, refs = [], [], [], []
    try:
        for k, (n, L) in enumerate(SHAPES):
            g = B.of_grid_create(n, L, 6, stream)
            grids.append(g)
            grid = O.Grid(n, L, 6)
            rho = W.random_field(grid.shape, seed=20 + k, kind="smooth") + 0.1 * W.random_field(grid.shape, seed=40 + k)
            rhos.append(torch.from_numpy(rho).cuda())
            phis.append(torch.zeros(grid.shape, dtype=torch.float64, device="cuda"))
            refs.append(O.poisson_solve(rho, grid))
        infos = B.of_poisson_solve_batched(grids, rhos, phis, _opts(1e-12, multigrid))
        for k in range(len(SHAPES)):
            got = phis[k].cpu().numpy()
            assert infos[k].rel_residual <= 1e-12, k
            assert np.max(np.abs(got - refs[k])) <= 1e-9 * np.max(np.abs(refs[k])), k
            assert abs(got.mean()) <= 1e-12 * np.max(np.abs(refs[k]))
            # the single-grid solver on the same cell (plain CG and multigrid PCG)
            for mg in (False, True):
                one = torch.zeros_like(phis[k])
                B.of_poisson_solve(grids[k], rhos[k], one, _opts(1e-12, mg))
                assert np.max(np.abs(one.cpu().numpy() - got)) <= 2e-9 * np.max(np.abs(refs[k]))
        # second call reuses the tuned blocking and the captured graphs
        for p in phis:
            p.zero_()
        B.of_poisson_solve_batched(grids, rhos, phis, _opts(1e-12, multigrid))
        for k in range(len(SHAPES)):
            assert np.max(np.abs(phis[k].cpu().numpy() - refs[k])) <= 1e-9 * np.max(np.abs(refs[k]))
    finally:
        for g in grids:
            B.of_grid_destroy(g)
