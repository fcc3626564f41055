"""Pins of the oracle's grid, FD stencils and exact periodic solves (Sec. 4)."""
from fractions import Fraction
from math import pi

import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_laplacian_weights_moment_conditions(N):
    # A 2N-th order central second difference must reproduce d^2/dx^2 x^{2j} at x = 0 for
    # j = 0..N exactly: 2 w_0 + 2 sum w_p = 0, 2 sum w_p p^2 h^2 = 2, 2 sum w_p p^{2j} = 0
    # (j = 2..N).  These N+1 linear conditions determine the N+1 weights uniquely.
    h = 0.37
    w = O.fd_laplacian_weights(N, h)
    assert abs(2 * w[0] + 2 * w[1:].sum()) < 1e-12 * abs(w[0])
    for j in range(1, N + 1):
        m = sum(2 * w[p] * (p * h) ** (2 * j) for p in range(1, N + 1))
        target = 2.0 if j == 1 else 0.0
        assert abs(m - target) < 1e-11 * max(1.0, sum(abs(2 * w[p] * (p * h) ** (2 * j)) for p in range(1, N + 1)))
    # order exactly 2N: the next moment is non-zero
    m = sum(2 * w[p] * (p * h) ** (2 * N + 2) for p in range(1, N + 1))
    assert abs(m) > 1e-6 * h ** (2 * N)


def test_laplacian_weights_twelfth_order_rationals():
    # N = 6 weights times h^2, from the closed form of Eq. FD:Laplacian evaluated by hand
    ref = [Fraction(-5369, 3600), Fraction(12, 7), Fraction(-15, 56), Fraction(10, 189),
           Fraction(-1, 112), Fraction(2, 1925), Fraction(-1, 16632)]
    w = O.fd_laplacian_weights(6, 1.0)
    for p in range(7):
        assert abs(w[p] - float(ref[p])) < 1e-15


@pytest.mark.parametrize("N", [1, 3, 6])
def test_gradient_weights_moment_conditions(N):
    h = 0.41
    w = O.fd_gradient_weights(N, h)
    for j in range(1, N + 1):
        m = sum(2 * w[p] * (p * h) ** (2 * j - 1) for p in range(1, N + 1))
        assert abs(m - (1.0 if j == 1 else 0.0)) < 1e-11 * max(1, sum(abs(2 * w[p] * (p * h) ** (2 * j - 1)) for p in range(1, N + 1)))


def _plane_wave(grid, m):
    n1, n2, n3 = grid.n
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    return np.exp(2j * pi * (m[0] * x / n1 + m[1] * y / n2 + m[2] * z / n3))


@pytest.mark.parametrize("n,N", [((8, 8, 8), 6), ((5, 6, 7), 6), ((12, 20, 9), 3), ((32, 32, 32), 6)])
def test_laplacian_symbol_plane_waves(n, N):
    grid = O.Grid(n, (7.6, 8.1, 6.9), N)
    sig = O.laplacian_symbol(grid)
    rng = np.random.default_rng(0)
    for _ in range(6):
        m = [int(rng.integers(0, n[d])) for d in range(3)]
        f = _plane_wave(grid, m)
        lf = O.laplacian(f, grid)
        expect = sig[m[2], m[1], m[0]] * f
        assert np.max(np.abs(lf - expect)) < 1e-12 * np.max(np.abs(sig))


def test_symbol_approximates_minus_k_squared():
    # sigma(k) = -|k|^2 (1 + O((kh)^{2N})) for small kh
    grid = O.Grid((64, 64, 64), (7.6, 7.6, 7.6), 6)
    sig = O.laplacian_symbol(grid)
    h = grid.h[0]
    for m in [1, 2, 4, 8]:
        k = 2 * pi * m / 7.6
        rel = abs(sig[0, 0, m] + k * k) / (k * k)
        assert rel < 2e-5 * (k * h) ** 12 + 1e-12


def test_laplacian_dense_matrix_by_index_loops():
    # Build the periodic FD Laplacian as a dense matrix with explicit modular index loops
    # (the definition of Eq. FD:Laplacian with the periodic wrap) and compare.
    for n, L, N in [((8, 8, 8), (7.6, 7.6, 7.6), 6), ((5, 6, 7), (5.0, 6.5, 7.2), 4)]:
        grid = O.Grid(n, L, N)
        n1, n2, n3 = n
        size = n1 * n2 * n3
        A = np.zeros((size, size))
        idx = lambda i, j, k: (i % n1) + n1 * ((j % n2) + n2 * (k % n3))
        ws = [O.fd_laplacian_weights(N, grid.h[d]) for d in range(3)]
        for k in range(n3):
            for j in range(n2):
                for i in range(n1):
                    row = idx(i, j, k)
                    for p in range(N + 1):
                        for sgn in (1, -1):
                            A[row, idx(i + sgn * p, j, k)] += ws[0][p]
                            A[row, idx(i, j + sgn * p, k)] += ws[1][p]
                            A[row, idx(i, j, k + sgn * p)] += ws[2][p]
        x = W.random_field(grid.shape, seed=3)
        y = O.laplacian(x, grid)
        assert np.allclose(y.ravel(), A @ x.ravel(), rtol=0, atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("N", [1, 2, 3])
def test_truncation_order(N):
    # error of L_h sin(2 pi x / L) against -(2 pi/L)^2 sin decreases like h^{2N}
    errs = []
    ns = [12, 24]
    for n in ns:
        grid = O.Grid((n, 4, 4), (7.6, 1.0, 1.0), N)
        x = np.arange(n) * grid.h[0]
        f = np.broadcast_to(np.sin(2 * pi * x / 7.6), grid.shape).copy()
        lf = O.laplacian(f, grid)
        errs.append(np.max(np.abs(lf + (2 * pi / 7.6) ** 2 * f)))
    rate = np.log(errs[0] / errs[1]) / np.log(2)
    assert abs(rate - 2 * N) < 0.15


def test_gradient_plane_wave():
    grid = O.Grid((10, 12, 14), (7.6, 7.0, 9.0), 6)
    m = (3, 5, 2)
    f = _plane_wave(grid, m)
    g = O.gradient(f, grid)
    for d in range(3):
        w = O.fd_gradient_weights(6, grid.h[d])
        th = 2 * pi * m[d] / grid.n[d]
        sym = 1j * sum(2 * w[p] * np.sin(p * th) for p in range(1, 7))
        assert np.max(np.abs(g[d] - sym * f)) < 1e-12 * np.max(np.abs(w)) * 12


def _dense_minus_laplacian(grid):
    size = grid.n[0] * grid.n[1] * grid.n[2]
    A = np.zeros((size, size))
    for c in range(size):
        e = np.zeros(size)
        e[c] = 1.0
        A[:, c] = -O.laplacian(e.reshape(grid.shape), grid).ravel()
    return A


def test_poisson_solve_matches_dense_pseudoinverse():
    grid = O.Grid((8, 8, 8), (7.6, 7.6, 7.6), 6)
    A = _dense_minus_laplacian(grid)
    rho = W.random_field(grid.shape, seed=5)
    phi = O.poisson_solve(rho, grid)
    rhs = 4 * pi * (rho - rho.mean()).ravel()
    ref = np.linalg.pinv(A) @ rhs
    ref -= ref.mean()
    assert np.max(np.abs(phi.ravel() - ref)) < 1e-10 * np.max(np.abs(ref))
    assert abs(phi.mean()) < 1e-14


def test_shifted_solve_matches_dense_complex():
    grid = O.Grid((8, 8, 8), (7.6, 7.6, 7.6), 6)
    A = _dense_minus_laplacian(grid)
    f = W.random_field(grid.shape, seed=6) + 1j * W.random_field(grid.shape, seed=7)
    scale, shift = 1 / 3.47, -0.470923 - 0.465392j
    W_ = O.solve_shifted_spectral(f, grid, scale, shift)
    ref = np.linalg.solve(scale * A + shift * np.eye(A.shape[0]), f.ravel())
    assert np.max(np.abs(W_.ravel() - ref)) < 1e-11 * np.max(np.abs(ref))


def test_poisson_of_gaussians_matches_analytic_series():
    # -(1/4pi) lap phi = b for Gaussian charges: continuum Fourier series
    # phi^(k) = 4 pi b^(k)/k^2, b^(k) = -Z e^{-k^2 s^2/2} sum_J e^{-i k R_J} / Omega.
    c = W.al4_displaced_cell(points_per_cell=32)
    grid = O.Grid(c.n, c.L, 6)
    b = O.pseudocharge(c.R, c.Z, c.sigma, c.rc, grid)
    phi = O.poisson_solve(b, grid)
    n = c.n[0]
    Lc = c.L[0]
    z, y, x = np.meshgrid(*(np.arange(n) * grid.h[0],) * 3, indexing="ij")
    ref = np.zeros(grid.shape)
    M = 8
    for m1 in range(-M, M + 1):
        for m2 in range(-M, M + 1):
            for m3 in range(-M, M + 1):
                if m1 == m2 == m3 == 0:
                    continue
                k = 2 * pi * np.array([m1, m2, m3]) / Lc
                k2 = k @ k
                sk = sum(np.exp(-1j * (k @ c.R[J])) for J in range(len(c.Z)))
                amp = 4 * pi * (-c.Z[0]) * np.exp(-k2 * c.sigma**2 / 2) * sk / (k2 * Lc**3)
                ref += (amp * np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))).real
    assert np.max(np.abs(phi - ref)) < 1e-6 * np.max(np.abs(ref))
