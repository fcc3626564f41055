"""GPU parity of the CUDA path (called through the C ABI) against the FP64 CPU oracle:
Laplacian, Poisson and shifted solves, pseudocharges, Hamiltonian, kernel potential, forces.

Tolerances: FP64 stencil and pointwise work 1e-13 relative (rounding order only); FP64
solves to relative residual 1e-13 agree with the exact discrete solution to 1e-10 relative;
FP32 sweeps agree to a few FP32 ulps of the stencil's absolute weight sum; mixed-precision
solves (FP32 inner, FP64 refinement) reach the same FP64 residual target.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    B.load()
    yield


class G:
    def __init__(self, n, L, N=6):
        self.n, self.L, self.N = tuple(n), tuple(L), N
        self.h = B.of_grid_create(n, L, N, torch.cuda.current_stream())
        self.grid = O.Grid(self.n, self.L, N)
        self.shape = self.grid.shape

    def __enter__(self):
        return self

    def __exit__(self, *a):
        B.of_grid_destroy(self.h)


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


LAP_CASES = [((32, 32, 32), (7.6, 7.6, 7.6), 6), ((5, 6, 7), (5.0, 6.5, 7.2), 6),
             ((8, 8, 8), (7.6, 7.6, 7.6), 6), ((33, 17, 40), (8.0, 4.1, 9.5), 3),
             ((12, 20, 9), (7.6, 8.1, 6.9), 1), ((96, 96, 96), (22.8, 22.8, 22.8), 6),
             ((70, 45, 3), (16.0, 10.0, 0.8), 6), ((1, 1, 16), (1.0, 1.0, 4.0), 3),
             ((36, 10, 13), (8.6, 2.4, 3.1), 6), ((44, 9, 5), (10.5, 2.1, 1.2), 1)]
# FP32: grids below 2^21 points with n1 % 4 == 0 and N in {1, 6} take the brick kernel
# (16 x 8 x 8 float2 units staged with their halo); the last two leave partial bricks in
# every direction, (5, 6, 7) and N = 3 take the general kernel
FP32_CASES = LAP_CASES[:6] + LAP_CASES[8:]


@pytest.mark.parametrize("n,L,N", LAP_CASES)
def test_laplacian_fp64(n, L, N):
    with G(n, L, N) as g:
        x = W.random_field(g.shape, seed=sum(n) + N)
        xd = dev(x)
        yd = torch.empty_like(xd)
        B.of_laplacian_apply(g.h, B.OF_F64, xd, yd)
        ref = O.laplacian(x, g.grid)
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.max(np.abs(host(yd) - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("n,L,N", FP32_CASES)
def test_laplacian_fp32(n, L, N):
    with G(n, L, N) as g:
        x = W.random_field(g.shape, seed=7).astype(np.float32)
        xd = dev(x, torch.float32)
        yd = torch.empty_like(xd)
        B.of_laplacian_apply(g.h, B.OF_F32, xd, yd)
        ref = O.laplacian(x.astype(np.float64), g.grid)
        wsum = sum(np.abs(O.fd_laplacian_weights(N, hd)).sum() * 2 for hd in g.grid.h)
        assert np.max(np.abs(host(yd) - ref)) <= 8 * 2**-24 * wsum * np.max(np.abs(x))


# grids of at least 2^21 points with even n1 take the FP32 fast-path sweep (float2 points, two
# rows per thread, 32 x 32 tiles); these sizes leave partial tiles in x and y
LARGE_CASES = [((136, 140, 120), (32.3, 33.25, 28.5)), ((160, 128, 104), (38.0, 30.4, 24.7))]


@pytest.mark.parametrize("n,L", LARGE_CASES)
def test_laplacian_fp32_large_grids(n, L):
    with G(n, L, 6) as g:
        x = W.random_field(g.shape, seed=9).astype(np.float32)
        xd = dev(x, torch.float32)
        yd = torch.empty_like(xd)
        B.of_laplacian_apply(g.h, B.OF_F32, xd, yd)
        ref = O.laplacian(x.astype(np.float64), g.grid)
        wsum = sum(np.abs(O.fd_laplacian_weights(6, hd)).sum() * 2 for hd in g.grid.h)
        assert np.max(np.abs(host(yd) - ref)) <= 8 * 2**-24 * wsum * np.max(np.abs(x))


# more fast-path grids, tiled whole by its 32 x 32 tiles: 128^3 exactly at the threshold, a
# non-cubic grid cut into several z chunks, and a z-thin grid whose register queue wraps in z
# more than once
WHOLE_TILE_CASES = [((128, 128, 128), (30.4, 30.4, 30.4)), ((320, 96, 80), (76.0, 22.8, 19.0)),
                    ((256, 1024, 9), (60.8, 243.2, 2.1375))]


@pytest.mark.parametrize("n,L", WHOLE_TILE_CASES)
def test_laplacian_fp32_whole_tile_grids(n, L):
    with G(n, L, 6) as g:
        x = W.random_field(g.shape, seed=11).astype(np.float32)
        xd = dev(x, torch.float32)
        yd = torch.full_like(xd, float("nan"))
        B.of_laplacian_apply(g.h, B.OF_F32, xd, yd)
        ref = O.laplacian(x.astype(np.float64), g.grid)
        wsum = sum(np.abs(O.fd_laplacian_weights(6, hd)).sum() * 2 for hd in g.grid.h)
        got = host(yd)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 8 * 2**-24 * wsum * np.max(np.abs(x))


@pytest.mark.parametrize("n,L", LARGE_CASES[:1])
def test_poisson_mixed_large_grid(n, L):
    # the mixed solve's FP32 Krylov and V-cycle sweeps run on the fast path at this size
    with G(n, L) as g:
        rho = W.random_field(g.shape, seed=3, kind="smooth") + 0.1 * W.random_field(g.shape, seed=4)
        ref = O.poisson_solve(rho, g.grid)
        phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        info = B.of_poisson_solve(g.h, dev(rho), phi, _opts(B.OF_F32, 1e-13))
        assert info.rel_residual <= 1e-13
        assert np.max(np.abs(host(phi) - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_laplacian_symbol_on_device():
    with G((24, 18, 30), (7.6, 6.0, 9.0), 6) as g:
        sig = O.laplacian_symbol(g.grid)
        m = (5, 3, 7)
        z, y, x = np.meshgrid(np.arange(30), np.arange(18), np.arange(24), indexing="ij")
        f = np.cos(2 * np.pi * (m[0] * x / 24 + m[1] * y / 18 + m[2] * z / 30))
        fd = dev(f)
        yd = torch.empty_like(fd)
        B.of_laplacian_apply(g.h, B.OF_F64, fd, yd)
        assert np.max(np.abs(host(yd) - sig[m[2], m[1], m[0]] * f)) < 1e-12 * abs(sig).max()


def _opts(prec, tol):
    o = B.of_default_solve_opts()
    o.tol = tol
    o.precision = prec
    return o


POISSON_CASES = [((32, 32, 32), (7.6, 7.6, 7.6)), ((24, 20, 28), (7.0, 6.0, 8.5)),
                 ((96, 96, 96), (22.8, 22.8, 22.8))]


@pytest.mark.parametrize("n,L", POISSON_CASES)
@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_poisson_matches_exact_discrete_solution(n, L, prec):
    with G(n, L) as g:
        rho = W.random_field(g.shape, seed=3, kind="smooth") + 0.1 * W.random_field(g.shape, seed=4)
        ref = O.poisson_solve(rho, g.grid)
        phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        info = B.of_poisson_solve(g.h, dev(rho), phi, _opts(prec, 1e-13))
        assert info.rel_residual <= 1e-13
        out = host(phi)
        assert abs(out.mean()) < 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(out - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_poisson_warm_start_and_zero_rhs():
    with G((16, 16, 16), (7.6, 7.6, 7.6)) as g:
        rho = W.random_field(g.shape, seed=5)
        ref = O.poisson_solve(rho, g.grid)
        phi = dev(ref)
        info = B.of_poisson_solve(g.h, dev(rho), phi, _opts(B.OF_F64, 1e-10))
        assert info.iterations <= 2
        zero = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        phi2 = dev(W.random_field(g.shape, seed=6))
        B.of_poisson_solve(g.h, zero, phi2, _opts(B.OF_F64, 1e-10))
        assert np.max(np.abs(host(phi2))) == 0.0


def test_poisson_iteration_limit_reports_enoconv():
    with G((32, 32, 32), (7.6, 7.6, 7.6)) as g:
        rho = W.random_field(g.shape, seed=8)
        phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        o = _opts(B.OF_F64, 1e-13)
        o.max_iter = 3
        info = B.of_poisson_solve(g.h, dev(rho), phi, o, allow=(B.OF_ENOCONV,))
        assert info.rel_residual > 1e-13
        assert "iterations" in B.of_last_error()


@pytest.mark.parametrize("n,L", [((32, 32, 32), (7.6, 7.6, 7.6)), ((20, 24, 18), (6.0, 7.0, 5.5)),
                                 ((96, 96, 96), (22.8, 22.8, 22.8))])
@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_kernel_solve_matches_exact_discrete_solution(n, L, prec):
    with G(n, L) as g:
        kf2 = Fn.kf2(3.0 * 4 * (L[0] * L[1] * L[2]) / 7.6**3, L[0] * L[1] * L[2])
        u = W.random_field(g.shape, seed=11, kind="smooth")
        f = -O.laplacian(u ** 0.92, g.grid) / kf2
        P = np.array(Fn.P00)
        Q = np.array(Fn.Q00)
        Wd = torch.zeros((2,) + g.shape + (2,), dtype=torch.float64, device="cuda")
        info = B.of_kernel_solve(g.h, dev(f), P, Q, kf2, Wd, _opts(prec, 1e-12))
        assert info.rel_residual <= 1e-12
        out = host(Wd)
        for s in range(2):
            ref = O.kernel_solve(f, g.grid, kf2, P[s], Q[s])
            got = out[s, ..., 0] + 1j * out[s, ..., 1]
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_kernel_solve_multigrid_cocg_cuts_iterations():
    # the mixed form preconditions COCG with a V-cycle of -L + |Q| kf2: same answer as plain
    # COCG (no_multigrid) in far fewer iterations
    n, L = (96, 96, 96), (22.8, 22.8, 22.8)
    with G(n, L) as g:
        kf2 = Fn.kf2(324.0, L[0] * L[1] * L[2])
        u = W.random_field(g.shape, seed=11, kind="smooth")
        f = -O.laplacian(u ** 0.92, g.grid) / kf2
        P, Q = np.array(Fn.P00), np.array(Fn.Q00)
        out = {}
        for mg in (0, 1):
            Wd = torch.zeros((2,) + g.shape + (2,), dtype=torch.float64, device="cuda")
            o = _opts(B.OF_F32, 1e-10)
            o.no_multigrid = 1 - mg
            info = B.of_kernel_solve(g.h, dev(f), P, Q, kf2, Wd, o)
            assert info.rel_residual <= 1e-10
            out[mg] = (host(Wd), info.iterations)
        scale = np.max(np.abs(out[0][0]))
        assert np.max(np.abs(out[1][0] - out[0][0])) <= 1e-8 * scale
        assert out[1][1] < 0.3 * out[0][1], (out[1][1], out[0][1])


@pytest.mark.parametrize("cell", [W.al4_cell(), W.al4_lr_cell(), W.al108_cell(),
                                  W.small_cell(n=(20, 14, 26), L=(7.0, 5.0, 9.0), seed=3)],
                         ids=["al4", "al4_lr", "al108", "ragged"])
def test_pseudocharge_and_self_energy(cell):
    with G(cell.n, cell.L) as g:
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        b = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        e = B.of_pseudocharge(g.h, sysd, b)
        ref = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, g.grid)
        assert np.max(np.abs(host(b) - ref)) <= 1e-13 * np.max(np.abs(ref))
        eref = O.self_energy(cell.R, cell.Z, cell.sigma, cell.rc, g.grid)
        assert abs(e - eref) <= 1e-12 * abs(eref)


def test_multigrid_solves_are_bitwise_reproducible():
    # the multigrid-preconditioned FP32 passes (Poisson and a shifted system) give the same bits
    # on repeated calls and on another handle.  This caught a data race: the first
    # post-smoothing step read the residual at its neighbours while other blocks rewrote it.
    cell = W.al108_cell()
    rho = torch.from_numpy(W.random_field(cell.shape, seed=5, kind="smooth")
                           + 0.1 * W.random_field(cell.shape, seed=6)).cuda()
    f = torch.from_numpy(W.random_field(cell.shape, seed=7, kind="smooth")).cuda()
    kf2 = Fn.kf2(cell.n_electrons, float(np.prod(cell.L)))
    fn = Fn.wt()
    P, Q = [complex(fn.P[4], fn.P[5])], [complex(fn.Q[4], fn.Q[5])]
    out = []
    for k in range(3):
        with G(cell.n, cell.L) as g:
            for rep in range(1 if k < 2 else 2):
                phi = torch.zeros_like(rho)
                B.of_poisson_solve(g.h, rho, phi, _opts(B.OF_F32, 1e-10))
                Wc = torch.zeros(cell.shape + (2,), dtype=torch.float64, device="cuda")
                B.of_kernel_solve(g.h, f, P, Q, kf2, Wc, _opts(B.OF_F32, 1e-10))
                out.append((phi, Wc))
    for phi, Wc in out[1:]:
        assert torch.equal(phi, out[0][0]) and torch.equal(Wc, out[0][1])


def test_pseudocharge_is_bitwise_reproducible():
    # every point of the nuclear charge is summed over the ions' images in one fixed order, so
    # two handles give the same bits (a scatter with atomics would not)
    for cell in (W.al108_cell(), W.al4_cell()):
        out = []
        for _ in range(2):
            with G(cell.n, cell.L) as g:
                b = torch.empty(g.shape, dtype=torch.float64, device="cuda")
                e = B.of_pseudocharge(g.h, B.make_system(cell.R, cell.Z, cell.sigma, cell.rc), b)
                out.append((b, e))
        assert torch.equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


@pytest.mark.parametrize("cell", [W.al4_displaced_cell(points_per_cell=24), W.al4_lr_cell(points_per_cell=20)],
                         ids=["al4d", "al4lr"])
def test_pseudocharge_from_the_potential(cell):
    # b_J = -(1/4pi) L_h V_J on each ion's widened box (Sec. 4), against the oracle's
    from oracle.pseudo import pseudocharge_fd
    with G(cell.n, cell.L) as g:
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc, b_from_potential=True)
        b = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        e = B.of_pseudocharge(g.h, sysd, b)
        ref, eref = pseudocharge_fd(cell.R, cell.Z, cell.sigma, cell.rc, g.grid)
        assert np.max(np.abs(host(b) - ref)) <= 1e-12 * np.max(np.abs(ref))
        assert abs(e - eref) <= 1e-12 * abs(eref)


@pytest.mark.parametrize("which", ["tfw", "wt"])
def test_hamiltonian_apply(which):
    with G((24, 28, 20), (7.6, 8.0, 6.5)) as g:
        u = 0.2 * W.random_field(g.shape, seed=1, kind="smooth")
        u[0, 0, :4] = 0.9       # a high-density region: the r_s < 1 branch of PZ
        phi = W.random_field(g.shape, seed=2)
        V = 0.3 * W.random_field(g.shape, seed=3)
        fn_d = Fn.tfw() if which == "tfw" else Fn.wt()
        fn_o = O.tfw_functional() if which == "tfw" else O.wt_functional()
        hu = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        B.of_hamiltonian_apply(g.h, fn_d, dev(u), dev(phi), dev(V), hu)
        ref = O.hamiltonian_apply(u, phi, V, g.grid, fn_o)
        assert np.max(np.abs(host(hu) - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_lr_potential(prec):
    cell = W.al4_lr_cell(points_per_cell=24)
    with G(cell.n, cell.L) as g:
        u = W.random_field(g.shape, seed=4, kind="smooth")
        u *= np.sqrt(cell.n_electrons / (g.grid.dV * np.sum(u * u)))
        kf2 = Fn.kf2(cell.n_electrons, g.grid.volume)
        v = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        T, info = B.of_lr_potential(g.h, Fn.wt(), kf2, dev(u), v, opts=_opts(prec, 1e-12))
        Vref, Tref, _, _ = O.lr_potential(u, g.grid, O.wt_functional(), kf2)
        assert np.max(np.abs(host(v) - Vref)) <= 1e-9 * np.max(np.abs(Vref))
        assert abs(T - Tref) <= 1e-9 * abs(Tref)


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_lr_potential_second_order_wgc(prec):
    # L = 2: 16 potentials (32 shifted solves) and the sum over m, n, p, q against the oracle
    cell = W.al4_lr_cell(points_per_cell=20)
    with G(cell.n, cell.L) as g:
        u = W.random_field(g.shape, seed=6, kind="smooth")
        u *= np.sqrt(cell.n_electrons / (g.grid.dV * np.sum(u * u)))
        kf2 = Fn.kf2(cell.n_electrons, g.grid.volume)
        fn = Fn.wgc()
        assert B.of_lr_workspace_fields(fn) == 32 and B.of_lr_workspace_fields(Fn.wt()) == 4
        v = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        T, info = B.of_lr_potential(g.h, fn, kf2, dev(u), v, opts=_opts(prec, 1e-12))
        Vref, Tref, _ = O.lr_potential_wgc(u, g.grid, O.wgc_functional(), kf2)
        assert np.max(np.abs(host(v) - Vref)) <= 1e-9 * np.max(np.abs(Vref))
        assert abs(T - Tref) <= 1e-9 * abs(Tref)
        assert info.iterations > 0


@pytest.mark.parametrize("cell", [W.al4_displaced_cell(), W.al108_cell()], ids=["al4d", "al108"])
def test_forces_for_given_potential(cell):
    with G(cell.n, cell.L) as g:
        phi = W.random_field(g.shape, seed=9, kind="smooth")
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        F = B.of_forces(g.h, sysd, None, dev(phi))
        ref = O.forces(phi, cell.R, cell.Z, cell.sigma, cell.rc, g.grid)
        assert np.max(np.abs(F - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_alu_peak_probe_gives_plausible_rates():
    # the roofline denominator of the FP64 stencil: a measured DFMA rate, between the FP64 rate
    # a Blackwell part could plausibly have and the FP32 rate, and an FP32 rate of the order of
    # 152 SMs x 128 lanes x 2 flops x ~2 GHz
    f64 = B.of_alu_peak(B.OF_PEAK_F64)
    f32 = B.of_alu_peak(B.OF_PEAK_F32)
    f32x2 = B.of_alu_peak(B.OF_PEAK_F32X2)
    assert 1e11 < f64 < f32
    assert 2e13 < f32 < 2e14
    assert 0.8 * f32 < f32x2 < 2.5 * f32
