"""The Poisson solve that allocates no device memory, for callers that cannot call
cudaMalloc (their allocator is not theirs to use, or device memory is reserved up front).

Called twice in a row through the C ABI on the same inputs, it must agree with the
allocating entry point of_poisson_solve (FP64) to the tolerance the Poisson tests use, and
with the exact discrete solution of the oracle; a second, different right-hand side checks
that nothing left in the shared scratch array from the previous call leaks into the next.
Collected last (file name) so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import binding as B, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _opts(tol):
    o = B.of_default_solve_opts()
    o.tol = tol
    o.precision = B.OF_F64
    return o


@pytest.mark.parametrize("n,L", [((32, 32, 32), (7.6, 7.6, 7.6)), ((24, 20, 28), (7.0, 6.0, 8.5))])
def test_noalloc_poisson_matches_allocating_entry_point(n, L):
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    grid = O.Grid(n, L, 6)
    stream = torch.cuda.current_stream()
    h = B.of_grid_create(n, L, 6, stream)
    try:
        for seed in (3, 4):
            rho = W.random_field(grid.shape, seed=seed, kind="smooth") + 0.1 * W.random_field(grid.shape, seed=seed + 10)
            rd = torch.from_numpy(rho).cuda()
            ref_phi = torch.zeros_like(rd)
            B.of_poisson_solve(h, rd, ref_phi, _opts(1e-13))
            ref = ref_phi.cpu().numpy()
            exact = O.poisson_solve(rho, grid)
            for call in range(2):
                phi = torch.zeros_like(rd)
                info = B.of_poisson_solve_noalloc(n, L, 6, stream, rd, phi, _opts(1e-13))
                got = phi.cpu().numpy()
                assert info.rel_residual <= 1e-13, (seed, call)
                assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref)), (seed, call)
                assert np.max(np.abs(got - exact)) <= 1e-10 * np.max(np.abs(exact)), (seed, call)
    finally:
        B.of_grid_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.OfError) as e:
        B.of_poisson_solve_noalloc((65, 64, 64), (7.6, 7.6, 7.6), 6, None, x, x, _opts(1e-10))
    assert "no-allocation limit" in str(e.value)
    o = _opts(1e-10)
    o.precision = B.OF_F32
    with pytest.raises(B.OfError):
        B.of_poisson_solve_noalloc((8, 8, 8), (7.6, 7.6, 7.6), 6, None, x, x, o)


def test_noalloc_repeated_calls_create_and_leak_nothing():
    # 200 calls: the library creates no buffer, stream, event or graph (its own resource
    # counter stays put) and the device's free memory does not move
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    n, L = (32, 32, 32), (7.6, 7.6, 7.6)
    grid = O.Grid(n, L, 6)
    rho = W.random_field(grid.shape, seed=5, kind="smooth")
    rd = torch.from_numpy(rho).cuda()
    phi = torch.zeros_like(rd)
    stream = torch.cuda.current_stream()
    B.of_poisson_solve_noalloc(n, L, 6, stream, rd, phi, _opts(1e-10))   # device address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = B.of_resource_count()
    for _ in range(200):
        phi.zero_()
        info = B.of_poisson_solve_noalloc(n, L, 6, stream, rd, phi, _opts(1e-10))
        assert info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert B.of_resource_count() == res0
    assert free1 == free0, (free0, free1)
    exact = O.poisson_solve(rho, grid)
    assert np.max(np.abs(phi.cpu().numpy() - exact)) <= 1e-8 * np.max(np.abs(exact))
