"""Failure paths of the C ABI, made without a GPU fault.

* Non-finite input (a NaN or an infinity planted on the host) must come back as OF_EINVAL
  with a message, never as a "converged" zero or garbage answer: a NaN compares false against
  every tolerance, so an unchecked solve would take it for a zero right-hand side.
* A Krylov breakdown must come back as OF_EBREAKDOWN.  The constructed case is a singular
  shifted system: Q = 0 and a constant right-hand side P * 1 on a grid with h = 1 and the
  order-2 stencil (weights -1, 1, centre -6: exact in binary), so L_h 1 = 0 exactly and
  p^T A p = 0 at the first COCG step.  The constant lies outside the range of L_h, so the
  system has no solution and breakdown is the right answer.
* The tensor-core kernels' bounded waits: with the wait limit set to zero every wait for an
  MMA completion gives up at once; the kernels then let the MMAs in flight finish, free their
  tensor memory and return, and the call reports OF_ETIMEOUT.  Afterwards, with the default
  limit, the same handle and grid give the same answer as before.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _grid(n=(16, 16, 16), L=(7.6, 7.6, 7.6), N=6):
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    return B.of_grid_create(n, L, N, torch.cuda.current_stream())


def _solve_opts(prec, tol=1e-10, no_multigrid=0):
    o = B.of_default_solve_opts()
    o.tol = tol
    o.precision = prec
    o.no_multigrid = no_multigrid
    return o


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_poisson_rejects_a_non_finite_right_hand_side(prec, bad):
    h = _grid()
    try:
        rho = torch.from_numpy(W.random_field((16, 16, 16), seed=1, kind="smooth")).cuda()
        rho[3, 4, 5] = bad
        phi = torch.zeros_like(rho)
        with pytest.raises(B.OfError) as e:
            B.of_poisson_solve(h, rho, phi, _solve_opts(prec))
        assert e.value.status == B.OF_EINVAL
        assert "not finite" in str(e.value)
        # the handle stays usable
        rho[3, 4, 5] = 0.0
        info = B.of_poisson_solve(h, rho, phi, _solve_opts(prec))
        assert info.rel_residual <= 1e-10
    finally:
        B.of_grid_destroy(h)


def test_poisson_rejects_a_non_finite_initial_guess():
    h = _grid()
    try:
        rho = torch.from_numpy(W.random_field((16, 16, 16), seed=1, kind="smooth")).cuda()
        phi = torch.zeros_like(rho)
        phi[0, 0, 7] = float("nan")
        with pytest.raises(B.OfError) as e:
            B.of_poisson_solve(h, rho, phi, _solve_opts(B.OF_F64))
        assert e.value.status == B.OF_EINVAL
        assert "non-finite residual" in str(e.value)
    finally:
        B.of_grid_destroy(h)


def test_noalloc_poisson_rejects_a_non_finite_right_hand_side():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    rho = torch.from_numpy(W.random_field((16, 16, 16), seed=1, kind="smooth")).cuda()
    rho[1, 2, 3] = float("nan")
    phi = torch.zeros_like(rho)
    with pytest.raises(B.OfError) as e:
        B.of_poisson_solve_noalloc((16, 16, 16), (7.6, 7.6, 7.6), 6, torch.cuda.current_stream(),
                                   rho, phi, _solve_opts(B.OF_F64))
    assert e.value.status == B.OF_EINVAL


def test_scf_rejects_a_non_finite_density():
    cell = W.al4_cell(points_per_cell=16)
    h = _grid(cell.n, cell.L)
    try:
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        u[2, 2, 2] = float("nan")
        phi = torch.zeros_like(u)
        with pytest.raises(B.OfError) as e:
            B.of_scf_ground_state(h, sysd, Fn.tfw(), B.of_default_scf_opts(), u, phi)
        assert e.value.status == B.OF_EINVAL
    finally:
        B.of_grid_destroy(h)


@pytest.mark.parametrize("prec,no_mg", [(B.OF_F64, 0), (B.OF_F32, 1)])
def test_singular_shifted_system_breaks_down(prec, no_mg):
    n = (8, 8, 8)
    h = _grid(n, (8.0, 8.0, 8.0), N=1)   # h = 1: exact order-2 weights
    try:
        f = torch.ones((8, 8, 8), dtype=torch.float64, device="cuda")
        Wc = torch.zeros((8, 8, 8, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(B.OfError) as e:
            B.of_kernel_solve(h, f, [1.0 + 0.0j], [0.0 + 0.0j], 1.0, Wc, _solve_opts(prec, no_multigrid=no_mg))
        assert e.value.status == B.OF_EBREAKDOWN, str(e.value)
        # a regular shifted system on the same handle still solves
        f2 = torch.from_numpy(W.random_field((8, 8, 8), seed=2)).cuda()
        Wc.zero_()
        info = B.of_kernel_solve(h, f2, [1.0 + 0.0j], [0.5 + 0.25j], 1.0, Wc,
                                 _solve_opts(prec, no_multigrid=no_mg))
        assert info.rel_residual <= 1e-10
    finally:
        B.of_grid_destroy(h)


def test_tensor_core_wait_limit_gives_a_timeout_status():
    n = (40, 36, 32)
    h = _grid(n, (0.2375 * 40, 0.2375 * 36, 0.2375 * 32))
    net = B.of_precond_create(W.initial_network(0))
    try:
        r = torch.from_numpy(W.random_field((32, 36, 40), seed=7).astype(np.float32)).cuda()
        z_ref = torch.empty_like(r)
        B.of_precond_apply(h, net, r, z_ref)
        for _ in range(2):   # twice: the first timeout left no tensor memory held
            B.of_precond_set_wait_limit(net, 0.0)
            z = torch.full_like(r, 7.0)
            with pytest.raises(B.OfError) as e:
                B.of_precond_apply(h, net, r, z)
            assert e.value.status == B.OF_ETIMEOUT, str(e.value)
            B.of_precond_set_wait_limit(net, 2.0)
            B.of_precond_apply(h, net, r, z)
            assert torch.equal(z, z_ref)
        with pytest.raises(B.OfError):
            B.of_precond_set_wait_limit(net, -1.0)
    finally:
        B.of_precond_destroy(net)
        B.of_grid_destroy(h)
