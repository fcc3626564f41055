"""Grid, order-2N finite differences and quadrature (Sec. 4 of arXiv:1412.8250).

Oracle (test infrastructure only).  Pins (tests/test_oracle_fd.py):
  * ``fd_laplacian_weights`` -- exact rational weights for N=6 typed from the closed form,
    weights sum to zero, the Fourier symbol of the stencil equals ``laplacian_symbol``
    exactly on every plane wave of several grids (including grids with fewer points than
    the stencil width, where indices wrap more than once), truncation error O(h^2N);
  * ``laplacian`` -- dense matrix built by explicit index loops on 8^3 / 5x6x7 grids;
  * ``gradient`` -- plane-wave symbol and the O(h^2N) truncation error;
  * ``poisson_solve`` / ``solve_shifted_spectral`` -- a dense brute-force solve of the
    same linear system on 8^3 grids (pseudo-inverse for the singular Poisson operator),
    and the analytic periodic potential of Gaussian charges.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import factorial, pi

import numpy as np


@dataclass(frozen=True)
class Grid:
    """Uniform periodic grid (Sec. 4): L_d = n_d h_d, points x = (i h1, j h2, k h3),
    0 <= i < n1 etc.  ``N`` is the half order: the FD stencils are of order 2N."""
    n: tuple
    L: tuple
    N: int = 6

    @property
    def h(self):
        return tuple(self.L[d] / self.n[d] for d in range(3))

    @property
    def dV(self):
        h = self.h
        return h[0] * h[1] * h[2]

    @property
    def volume(self):
        return self.L[0] * self.L[1] * self.L[2]

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


# numpy axis of each cartesian direction for arrays of shape (n3, n2, n1)
_AXIS = (2, 1, 0)


def fd_laplacian_weights(N: int, h: float) -> np.ndarray:
    """Weights w_0..w_N of the order-2N central second difference (Eq. FD:Laplacian):
    w_0 = -(1/h^2) sum_{q=1}^N 1/q^2,
    w_p = 2 (-1)^{p+1} (N!)^2 / (h^2 p^2 (N-p)! (N+p)!),  p = 1..N."""
    w = np.zeros(N + 1)
    w[0] = -sum(1.0 / q**2 for q in range(1, N + 1)) / h**2
    for p in range(1, N + 1):
        w[p] = (2.0 * (-1) ** (p + 1) * factorial(N) ** 2
                / (h**2 * p**2 * factorial(N - p) * factorial(N + p)))
    return w


def fd_gradient_weights(N: int, h: float) -> np.ndarray:
    """Weights w~_1..w~_N of the order-2N central first difference (Eq.
    gradient:approximate): w~_p = (-1)^{p+1} (N!)^2 / (h p (N-p)! (N+p)!).  Index 0 unused."""
    w = np.zeros(N + 1)
    for p in range(1, N + 1):
        w[p] = ((-1) ** (p + 1) * factorial(N) ** 2
                / (h * p * factorial(N - p) * factorial(N + p)))
    return w


def laplacian(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Order-2N FD Laplacian with periodic index wrap (Eq. FD:Laplacian and the periodic
    boundary treatment at the end of Sec. 4): for each axis d,
    sum_{p=0}^N w_p (f(i + p e_d) + f(i - p e_d)), indices taken modulo n_d."""
    out = np.zeros_like(f, dtype=np.result_type(f, np.float64))
    for d in range(3):
        w = fd_laplacian_weights(grid.N, grid.h[d])
        ax = _AXIS[d]
        for p in range(0, grid.N + 1):
            out += w[p] * (np.roll(f, -p, axis=ax) + np.roll(f, p, axis=ax))
    return out


def gradient(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Order-2N FD gradient with periodic wrap (Eq. gradient:approximate); returns an
    array of shape (3,) + f.shape, component d along e_d."""
    g = np.zeros((3,) + f.shape, dtype=np.result_type(f, np.float64))
    for d in range(3):
        w = fd_gradient_weights(grid.N, grid.h[d])
        ax = _AXIS[d]
        for p in range(1, grid.N + 1):
            g[d] += w[p] * (np.roll(f, -p, axis=ax) - np.roll(f, p, axis=ax))
    return g


def integrate(f: np.ndarray, grid: Grid) -> float:
    """Piecewise-constant quadrature (Eq. IntApprox): int f ~ h1 h2 h3 sum f."""
    return float(grid.dV * np.sum(f))


def laplacian_symbol(grid: Grid) -> np.ndarray:
    """Eigenvalues of the periodic FD Laplacian on the discrete Fourier modes
    exp(2 pi i m_d x_d / L_d): sigma(m) = sum_d [2 w_0 + 2 sum_p w_p cos(2 pi m_d p / n_d)].
    Returned with numpy shape (n3, n2, n1) in numpy.fft frequency order."""
    parts = []
    for d in range(3):
        n = grid.n[d]
        w = fd_laplacian_weights(grid.N, grid.h[d])
        m = np.arange(n)
        s = 2.0 * w[0] + sum(2.0 * w[p] * np.cos(2.0 * pi * m * p / n)
                             for p in range(1, grid.N + 1))
        parts.append(s)
    s1, s2, s3 = parts
    return s3[:, None, None] + s2[None, :, None] + s1[None, None, :]


def solve_shifted_spectral(rhs: np.ndarray, grid: Grid, scale: float, shift: complex):
    """Exact solution of (-scale * L_h + shift) W = rhs on the periodic grid.

    L_h is a circulant, so the discrete Fourier transform diagonalises it with the
    eigenvalues ``laplacian_symbol``; the solution is W^ = rhs^ / (-scale sigma + shift).
    This is the definition of the discrete solution that the Krylov solvers approximate.
    For shift == 0 the constant mode is projected out (mean-zero solution)."""
    sig = laplacian_symbol(grid)
    denom = -scale * sig + shift
    rh = np.fft.fftn(rhs)
    if shift == 0:
        rh.flat[0] = 0.0
        denom.flat[0] = 1.0
    W = np.fft.ifftn(rh / denom)
    if np.isrealobj(rhs) and np.isreal(shift):
        return W.real
    return W


def poisson_solve(rho: np.ndarray, grid: Grid) -> np.ndarray:
    """Periodic Poisson problem of Eq. Poisson, -(1/4pi) L_h phi = rho, with the mean of
    the right-hand side removed and int phi = 0 enforced (Sec. 4)."""
    rhs = 4.0 * pi * (rho - rho.mean())
    phi = solve_shifted_spectral(rhs, grid, 1.0, 0.0)
    return phi - phi.mean()
