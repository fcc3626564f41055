"""The 864-atom size: a 6x6x6 FCC cell's 192^3 grid (7.1 M points, h = 0.2375 bohr), on which
the learned preconditioner is measured against Jacobi CG.  Every solver form of the Poisson
system (Sec. 3.3.1) and of a shifted kernel system (Sec. 3.1) is run to the stopping test on
the true FP64 residual and compared element by element with the oracle's exact discrete
solution (FFT diagonalisation of the same order-12 operator) of the same seeded right-hand side.

The network here has the seeded initial weights (untrained): whatever it proposes, the flexible
solvers accept a direction only when it passes the angle test and stop on the true residual, so
the answer must be the oracle's either way.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
N = (192, 192, 192)
L = tuple(0.2375 * n for n in N)


def _opts(prec, no_mg, tol, net=None):
    o = B.of_default_solve_opts()
    o.tol, o.precision, o.no_multigrid, o.inner_tol = tol, prec, no_mg, 1e-4
    if net is not None:
        o.precond, o.precond_theta = net, 0.3
    return o


@pytest.fixture(scope="module")
def grid():
    h = B.of_grid_create(N, L, 6, torch.cuda.current_stream())
    yield h, O.Grid(N, L, 6)
    B.of_grid_destroy(h)


@pytest.fixture(scope="module")
def poisson_case(grid):
    g = grid[1]
    rho = (W.random_field(g.shape, seed=61, kind="smooth") - 2.0
           + 0.3 * W.random_field(g.shape, seed=62))
    return rho, O.poisson_solve(rho, g)


@pytest.fixture(scope="module")
def shifted_case(grid):
    # the WT kernel's second shift (Q = 0.066 - 0.260i), the right-hand side of the m = n = 0
    # form of Sec. 3.1 built from a smooth positive seeded field standing in for u^{2 alpha}
    g = grid[1]
    fn = Fn.wt()
    Pk, Qk = complex(fn.P[4], fn.P[5]), complex(fn.Q[4], fn.Q[5])
    kf2 = Fn.kf2(3.0 * 864, float(np.prod(L)))
    q = 1.0 + 0.5 * W.random_field(g.shape, seed=47, kind="smooth")
    f = -O.laplacian(q, g) / kf2
    return f, Pk, Qk, kf2, O.kernel_solve(f, g, kf2, Pk, Qk)


@pytest.mark.parametrize("form", ["jacobi_cg_mixed", "learned_fcg_mixed", "plain_cg_f64",
                                  "multigrid_pcg_mixed"])
def test_poisson_192_every_form_against_the_exact_solution(grid, poisson_case, form):
    h, g = grid
    rho, ref = poisson_case
    net = B.of_precond_create(W.initial_network(0)) if form == "learned_fcg_mixed" else None
    try:
        o = {"jacobi_cg_mixed": _opts(B.OF_F32, 1, 1e-12),
             "learned_fcg_mixed": _opts(B.OF_F32, 1, 1e-12, net),
             "plain_cg_f64": _opts(B.OF_F64, 1, 1e-12),
             "multigrid_pcg_mixed": _opts(B.OF_F32, 0, 1e-12)}[form]
        phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        info = B.of_poisson_solve(h, torch.from_numpy(rho).cuda(), phi, o)
    finally:
        if net is not None:
            B.of_precond_destroy(net)
    assert info.rel_residual <= 1e-12
    assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("form", ["plain_cocg_mixed", "learned_fgmres_mixed", "plain_cocg_f64",
                                  "multigrid_pcocg_mixed"])
def test_shifted_192_every_form_against_the_exact_solution(grid, shifted_case, form):
    h, g = grid
    f, Pk, Qk, kf2, ref = shifted_case
    net = None
    if form == "learned_fgmres_mixed":
        net = B.of_precond_create(W.initial_network(4))
        B.of_precond_set_shift(net, kf2 * abs(Qk))
    try:
        o = {"plain_cocg_mixed": _opts(B.OF_F32, 1, 1e-10),
             "learned_fgmres_mixed": _opts(B.OF_F32, 1, 1e-10, net),
             "plain_cocg_f64": _opts(B.OF_F64, 1, 1e-10),
             "multigrid_pcocg_mixed": _opts(B.OF_F32, 0, 1e-10)}[form]
        Wc = torch.zeros(g.shape + (2,), dtype=torch.float64, device="cuda")
        info = B.of_kernel_solve(h, torch.from_numpy(f).cuda(), [Pk], [Qk], kf2, Wc, o)
    finally:
        if net is not None:
            B.of_precond_destroy(net)
    w = Wc.cpu().numpy()
    assert info.rel_residual <= 1e-10
    assert np.abs(w[..., 0] + 1j * w[..., 1] - ref).max() <= 1e-9 * np.abs(ref).max()
