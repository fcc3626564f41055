"""Pins of the oracle's kernel (linear-response) term: shifted solves and V_LR (Sec. 3.1, App. A)."""
from math import pi

import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W


def test_table_sum_rule_and_conjugates():
    fn = O.wt_functional()
    assert abs(sum(fn.P).imag) < 1e-15 and abs(sum(fn.Q).imag) < 1e-15
    # K(s -> infinity) = sum_r P_r = 2 Re(P_1 + P_3) = -8/5 (large-eta limit of the
    # Lindhard response minus TF and vW), which the printed table satisfies to 6 digits
    assert abs(sum(fn.P).real + 1.6) < 1e-6
    assert fn.P[1] == np.conj(fn.P[0]) and fn.Q[3] == np.conj(fn.Q[2])


def test_plane_wave_closed_form():
    grid = O.Grid((16, 12, 10), (7.6, 6.0, 5.5), 6)
    kf2 = 3.4742
    sig = O.laplacian_symbol(grid)
    m = (3, 2, 1)
    z, y, x = np.meshgrid(np.arange(10), np.arange(12), np.arange(16), indexing="ij")
    g = np.cos(2 * pi * (m[0] * x / 16 + m[1] * y / 12 + m[2] * z / 10))
    f = -O.laplacian(g, grid) / kf2
    s = -sig[m[2], m[1], m[0]] / kf2
    for P, Q in zip(O.wt_functional().P, O.wt_functional().Q):
        V = O.kernel_solve(f, grid, kf2, P, Q)
        assert np.max(np.abs(V - P * s / (s + Q) * g)) < 1e-12


def test_conjugate_shifts_give_conjugate_solutions():
    grid = O.Grid((10, 10, 10), (7.6, 7.6, 7.6), 6)
    f = W.random_field(grid.shape, seed=2)
    fn = O.wt_functional()
    for r in (0, 2):
        a = O.kernel_solve(f, grid, 3.0, fn.P[r], fn.Q[r])
        b = O.kernel_solve(f, grid, 3.0, fn.P[r + 1], fn.Q[r + 1])
        assert np.max(np.abs(b - np.conj(a))) < 1e-13 * np.max(np.abs(a))


def _smooth_u(grid, Ne, seed=1):
    u = W.random_field(grid.shape, seed=seed, kind="smooth")
    return u * np.sqrt(Ne / (grid.dV * np.sum(u * u)))


def test_kernel_symmetry_and_energy_derivative():
    grid = O.Grid((12, 12, 12), (7.6, 7.6, 7.6), 6)
    fn = O.wt_functional()
    Ne = 12.0
    kf2 = O.kernel.kf2_of(Ne, grid.volume)
    u = _smooth_u(grid, Ne)
    V, T, Va, Vb = O.lr_potential(u, grid, fn, kf2)
    a = grid.dV * np.sum(u ** (2 * fn.alpha) * Vb)
    b = grid.dV * np.sum(u ** (2 * fn.beta) * Va)
    assert abs(a - b) < 1e-12 * abs(a)
    assert abs(T - O.C_F * a) < 1e-12 * abs(T)
    # V_LR = dT_LR / d rho: directional derivative along v
    v = W.random_field(grid.shape, seed=9)
    e = 1e-5
    dT = (O.lr_potential(u + e * v, grid, fn, kf2)[1] - O.lr_potential(u - e * v, grid, fn, kf2)[1]) / (2 * e)
    assert abs(dT - grid.dV * np.sum(V * 2 * u * v)) < 1e-7 * abs(dT)


def test_uniform_density_gives_zero_kernel_potential():
    grid = O.Grid((8, 8, 8), (7.6, 7.6, 7.6), 6)
    u = np.full(grid.shape, 0.165)
    V, T, _, _ = O.lr_potential(u, grid, O.wt_functional(), 3.47)
    assert np.max(np.abs(V)) < 1e-12 and abs(T) < 1e-12
