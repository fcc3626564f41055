"""Pins of the oracle's second-order (L = 2, WGC) kernel term: the coefficients C_mnpq of the
Taylor expansion of the density-dependent kernel (Sec. 2), the local potentials and energy of
Eq. VLinearResponse:local and the T_LR expression after it (Sec. 3.1), with App. A's table."""
import numpy as np
import pytest

import oracle as O
from paper_1412_8250_gb300 import workloads as W

GRID = ((12, 10, 14), (7.6, 6.3, 8.9))


def _setup(seed=1):
    grid = O.Grid(GRID[0], GRID[1], 6)
    kf2 = O.kf2_of(12.0, grid.volume)
    rho_bar = O.rho_bar_of(kf2)
    # a positive density near rho_bar with smooth variations of ~30 %
    rho = rho_bar * (0.7 + 0.3 * W.random_field(grid.shape, seed=seed, kind="smooth")
                     / W.random_field(grid.shape, seed=seed, kind="smooth").mean())
    return grid, kf2, rho_bar, np.sqrt(rho)


def test_rho_bar_round_trip():
    grid = O.Grid(GRID[0], GRID[1], 6)
    kf2 = O.kf2_of(12.0, grid.volume)
    assert abs(O.rho_bar_of(kf2) - 12.0 / grid.volume) < 1e-15 * 12.0 / grid.volume


@pytest.mark.parametrize("m,n", [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1)])
def test_c_mnpq_is_the_binomial_expansion(m, n):
    # sum_pq C_mnpq a^{m-p} b^{n-q} = ((a - rb) / rb)^m ((b - rb) / rb)^n / (m! n!): the
    # expansion of (rho - rho_bar)^m (rho' - rho_bar)^n that C_mnpq collects (Sec. 2)
    rng = np.random.default_rng(m * 7 + n)
    rb = 0.027
    for a, b in rng.uniform(0.005, 0.06, size=(5, 2)):
        lhs = sum(O.c_mnpq(m, n, p, q, rb) * a ** (m - p) * b ** (n - q)
                  for p in range(m + 1) for q in range(n + 1))
        fact = [1, 1, 2][m] * [1, 1, 2][n]
        rhs = ((a - rb) / rb) ** m * ((b - rb) / rb) ** n / fact
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_kernel_classes_follow_the_table_symmetry():
    assert O.kernel_class(1, 0) == O.kernel_class(0, 1) == "10"
    assert O.kernel_class(2, 0) == O.kernel_class(0, 2) == "20"
    fn = O.wgc_functional()
    assert fn.L == 2 and set(fn.K) == {"10", "20", "11"}
    for c, (P, Q) in fn.K.items():
        assert P[1] == np.conj(P[0]) and P[3] == np.conj(P[2])
        assert Q[1] == np.conj(Q[0]) and Q[3] == np.conj(Q[2])
        assert P[0] == O.WGC_TABLE[c]["P"][0] and Q[2] == O.WGC_TABLE[c]["Q"][1]


def test_each_class_is_a_symmetric_kernel():
    # int u^{2(k1+alpha)} (K_c u^{2(k2+beta)}) = int u^{2(k2+beta)} (K_c u^{2(k1+alpha)}): K_mn
    # depends on |x - x'| only.  The check would fail for a solve built from the other
    # exponent's power (the swapped labels of the Helmholtz equations).
    grid, kf2, rho_bar, u = _setup()
    fn = O.wgc_functional()
    _, _, pots = O.lr_potential_wgc(u, grid, fn, kf2)
    for (c, e, k) in pots:
        if e != "alpha":
            continue
        for k2 in range(3):
            if (c, "beta", k2) not in pots:
                continue
            lhs = np.sum(u ** (2 * (k + fn.alpha)) * pots[(c, "beta", k2)])
            rhs = np.sum(u ** (2 * (k2 + fn.beta)) * pots[(c, "alpha", k)])
            assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-30), (c, k, k2)


def test_v_lr_is_the_density_derivative_of_t_lr():
    # V_LR = dT_LR / d rho: central differences of T_LR along a smooth direction.  A dropped
    # term, a wrong (m - p + alpha) factor or a wrong power in V_LR fails this.
    grid, kf2, rho_bar, u = _setup(seed=3)
    fn = O.wgc_functional()
    V, T, _ = O.lr_potential_wgc(u, grid, fn, kf2)
    delta = rho_bar * (W.random_field(grid.shape, seed=9, kind="smooth") - 1.0)

    def central(eps):
        Tp = O.lr_potential_wgc(np.sqrt(u * u + eps * delta), grid, fn, kf2)[1]
        Tm = O.lr_potential_wgc(np.sqrt(u * u - eps * delta), grid, fn, kf2)[1]
        return (Tp - Tm) / (2 * eps)

    # Richardson: the O(eps^2) error of the central difference cancels (measured: 4.8e-6
    # relative at eps = 1e-4 alone, shrinking as eps^2)
    fd = (4.0 * central(1e-4) - central(2e-4)) / 3.0
    exact = grid.dV * float(np.sum(V * delta))
    assert abs(fd - exact) <= 1e-8 * abs(exact), (fd, exact)


def test_uniform_density_closed_form():
    # at rho = rho_bar every T_LR term vanishes (the m = n = 0 right-hand side is L_h of a
    # constant; the others carry (rho - rho_bar)^m) and only the first-order terms (1,0),
    # (0,1) survive in V_LR: V_LR = 2 C_F rho_bar^{alpha+beta-1} kappa_10 with kappa_10 =
    # sum_r Re(P_10r / Q_10r), the zero-wavenumber response of K_10.
    grid = O.Grid((8, 8, 8), (7.6, 7.6, 7.6), 6)
    kf2 = O.kf2_of(12.0, grid.volume)
    rb = O.rho_bar_of(kf2)
    fn = O.wgc_functional()
    u = np.full(grid.shape, np.sqrt(rb))
    V, T, _ = O.lr_potential_wgc(u, grid, fn, kf2)
    P, Q = fn.K["10"]
    kappa = sum((P[r] / Q[r]).real for r in range(4))
    ref = 2 * O.C_F * rb ** (fn.alpha + fn.beta - 1.0) * kappa
    # kappa_10 nearly vanishes (the fit's zero-wavenumber response); the bar is relative to
    # the size of the terms that cancel in it
    scale = 2 * O.C_F * rb ** (fn.alpha + fn.beta - 1.0) * sum(abs(P[r] / Q[r]) for r in range(4))
    assert abs(T) <= 1e-14
    assert np.max(np.abs(V - ref)) <= 1e-13 * scale


def test_zero_density_dependence_reduces_to_l0():
    grid, kf2, rho_bar, u = _setup(seed=5)
    fn = O.wgc_functional()
    for c in fn.K:
        fn.K[c] = (tuple(0j for _ in range(4)), fn.K[c][1])
    V2, T2, _ = O.lr_potential_wgc(u, grid, fn, kf2)
    V0, T0, _, _ = O.lr_potential(u, grid, O.wt_functional(), kf2)
    assert abs(T2 - T0) <= 1e-13 * abs(T0)
    assert np.max(np.abs(V2 - V0)) <= 1e-13 * np.max(np.abs(V0))


def test_lr_potential_dispatches_on_l():
    grid, kf2, rho_bar, u = _setup(seed=7)
    V, T, Va, Vb = O.lr_potential(u, grid, O.wgc_functional(), kf2)
    V2, T2, pots = O.lr_potential_wgc(u, grid, O.wgc_functional(), kf2)
    assert T == T2 and np.array_equal(V, V2)
    assert np.array_equal(Va, pots[("00", "alpha", 0)])
