"""Pins of the oracle's Hamiltonian, energy, NLCG, Anderson mixing and fixed point
(Sec. 3.3.1, App. C, App. D)."""
from math import pi, sqrt

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O
from oracle.scf import inner
from paper_1412_8250_gb300 import workloads as W


def _setup(cell, N=6):
    grid = O.Grid(cell.n, cell.L, N)
    b = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    return grid, b, O.poisson_solve(b, grid)


def _u(grid, Ne, seed=1):
    u = W.random_field(grid.shape, seed=seed, kind="smooth")
    return u * np.sqrt(Ne / (grid.dV * np.sum(u * u)))


@pytest.mark.parametrize("fn", [O.tfw_functional(), O.wt_functional()])
def test_energy_gradient_is_2dV_Hu(fn):
    cell = W.small_cell(n=(10, 11, 12), L=(7.0, 7.6, 8.2), sigma=1.0, rc=6.0, seed=3)
    grid, b, _ = _setup(cell)
    Ne = cell.n_electrons
    u = _u(grid, Ne)
    V_LR = 0.3 * W.random_field(grid.shape, seed=4)
    # include an r_s < 1 region so both PZ branches are exercised
    u[0, 0, :3] = 0.9
    energy = lambda w: O.inner_energy(w, O.poisson_solve(w * w + b, grid), b, V_LR, grid, fn)
    phi = O.poisson_solve(u * u + b, grid)
    Hu = O.hamiltonian_apply(u, phi, V_LR, grid, fn)
    v = W.random_field(grid.shape, seed=5)
    e = 1e-5
    fd = (energy(u + e * v) - energy(u - e * v)) / (2 * e)
    assert abs(fd - 2 * grid.dV * np.sum(Hu * v)) < 1e-7 * abs(fd)


def test_line_energy_by_linearity_equals_fresh_poisson():
    cell = W.small_cell(n=(12, 12, 12), seed=2)
    grid, b, phib = _setup(cell)
    Ne = cell.n_electrons
    fn = O.tfw_functional()
    u = _u(grid, Ne)
    d = W.random_field(grid.shape, seed=8)
    V = np.zeros(grid.shape)
    phi = O.poisson_solve(u * u + b, grid)
    pud, pdd = O.poisson_solve(u * d, grid), O.poisson_solve(d * d, grid)
    for s in [0.01, -0.2, 0.7]:
        w = u + s * d
        c2 = Ne / inner(w, w, grid)
        us = sqrt(c2) * w
        phis = c2 * (phi - phib + 2 * s * pud + s * s * pdd) + phib
        direct = O.poisson_solve(us * us + b, grid)
        assert np.max(np.abs(phis - direct)) < 1e-11 * np.max(np.abs(direct))


def test_nlcg_reaches_the_lbfgs_minimum():
    cell = W.small_cell(n=(10, 10, 10), sigma=1.0, rc=6.0, seed=11)
    grid, b, phib = _setup(cell)
    Ne = cell.n_electrons
    fn = O.tfw_functional()
    V = np.zeros(grid.shape)
    u0 = np.full(grid.shape, sqrt(Ne / grid.volume))
    u, phi, info = O.nlcg(u0, V, b, phib, grid, fn, Ne, tol=1e-7, max_iter=3000)
    assert info.converged
    e_nlcg = O.inner_energy(u, phi, b, V, grid, fn)
    assert abs(inner(u, u, grid) - Ne) < 1e-10 * Ne
    assert u.min() > 0

    def f(w):
        w = w.reshape(grid.shape)
        nw = sqrt(inner(w, w, grid))
        us = sqrt(Ne) * w / nw
        ph = O.poisson_solve(us * us + b, grid)
        E = O.inner_energy(us, ph, b, V, grid, fn)
        gu = 2 * grid.dV * O.hamiltonian_apply(us, ph, V, grid, fn)
        gw = (sqrt(Ne) / nw) * (gu - us * np.sum(gu * us) * grid.dV / Ne)
        return E, gw.ravel()

    res = minimize(f, u0.ravel(), jac=True, method="L-BFGS-B",
                   options=dict(maxiter=5000, gtol=1e-12, ftol=1e-16, maxcor=30))
    assert abs(res.fun - e_nlcg) < 1e-9 * abs(e_nlcg)
    w = res.x.reshape(grid.shape)
    ul = sqrt(Ne) * w / sqrt(inner(w, w, grid))
    assert np.max(np.abs(ul - u)) < 1e-4 * u.max()


def _gmres_iterate(A, rhs, x0, k):
    r0 = rhs - A @ x0
    if k == 0:
        return x0
    K = [r0]
    for _ in range(k - 1):
        K.append(A @ K[-1])
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    y = np.linalg.lstsq(A @ Q, r0, rcond=None)[0]
    return x0 + Q @ y


def test_anderson_equals_gmres_on_linear_fixed_point():
    # Walker & Ni (2011): for g(x) = Gx + c, Anderson with unbounded history and zeta = 1
    # satisfies x_{k+1}^AA = g(x_k^GMRES) for (I - G) x = c.
    rng = np.random.default_rng(0)
    n = 24
    G = rng.normal(size=(n, n))
    G *= 0.8 / np.max(np.abs(np.linalg.eigvals(G)))
    c = rng.normal(size=n)
    x0 = rng.normal(size=n)
    A = np.eye(n) - G
    Vh, fh = [x0], [G @ x0 + c - x0]
    for k in range(8):
        x_next = O.anderson_update(Vh, fh, 1.0, 100)
        ref = G @ _gmres_iterate(A, c, x0, k) + c
        assert np.max(np.abs(x_next - ref)) < 1e-9 * np.max(np.abs(ref))
        Vh.append(x_next)
        fh.append(G @ x_next + c - x_next)


def test_anderson_limited_history_and_damping_solve_linear_problem():
    rng = np.random.default_rng(1)
    n = 30
    G = rng.normal(size=(n, n))
    G = G + G.T
    G *= 0.9 / np.max(np.abs(np.linalg.eigvalsh(G)))
    c = rng.normal(size=n)
    x = np.zeros(n)
    Vh, fh = [], []
    for k in range(200):
        f = G @ x + c - x
        Vh.append(x)
        fh.append(f)
        if np.linalg.norm(f) < 1e-12:
            break
        x = O.anderson_update(Vh, fh, 0.3, 7)
    assert np.linalg.norm(G @ x + c - x) < 1e-10


@pytest.mark.slow
def test_fixed_point_ground_state_wt_small():
    cell = W.al4_lr_cell(points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    res = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(),
                             nlcg_tol=1e-8, fp_tol=1e-6, anderson_m=7, zeta=0.3)
    assert res.fp_errors[-1] < 1e-6
    # at the fixed point, u is the ground state of the full functional: the gradient with
    # the self-consistent V_LR vanishes
    b = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    kf2 = O.kf2_of(cell.n_electrons, grid.volume)
    V, T, _, _ = O.lr_potential(res.u, grid, O.wt_functional(), kf2)
    Hu = O.hamiltonian_apply(res.u, res.phi, V, grid, O.wt_functional())
    eta = inner(res.u, Hu, grid) / cell.n_electrons
    r = Hu - eta * res.u
    assert sqrt(inner(r, r, grid) / cell.n_electrons) < 1e-5


@pytest.mark.slow
def test_fixed_point_on_u_reaches_the_same_ground_state():
    # Sec. 5.3 compares Anderson mixing of V_LR (the method) with mixing of u; both fixed
    # points are the ground state of the full functional, so the energies agree
    cell = W.al4_lr_cell(points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    kw = dict(nlcg_tol=1e-8, fp_tol=1e-7, anderson_m=3, zeta=1.0)
    rv = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(), **kw)
    ru = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(),
                            fixed_point="u", **kw)
    assert ru.fp_errors[-1] < 1e-7 and rv.fp_errors[-1] < 1e-7
    assert abs(ru.energy - rv.energy) / cell.n_atoms < 1e-9
    assert np.max(np.abs(ru.u - rv.u)) < 1e-5 * np.max(rv.u)


def test_vw_energy_gradient_form_plane_wave_and_limit():
    # (lam/2) int |grad_h u|^2 for u = cos(2 pi m x / L): each mode contributes its FD symbol
    # squared, (sum_p 2 w~_p sin(2 pi m p / n))^2 / 2 per unit volume (Eq. gradient:approximate)
    grid = O.Grid((16, 12, 10), (7.6, 6.0, 5.5), 6)
    z, y, x = np.meshgrid(np.arange(10), np.arange(12), np.arange(16), indexing="ij")
    m = 3
    u = np.cos(2 * pi * m * x / 16)
    fn = O.tfw_functional()
    zero = np.zeros(grid.shape)
    _, tg = O.ground_state_energy(u, zero, zero, grid, fn, 0.0, 0.0, 0.0, vw_energy="gradient")
    w = O.fd_gradient_weights(6, grid.h[0])
    sym = sum(2 * w[p] * np.sin(2 * pi * m * p / 16) for p in range(1, 7))
    ref = 0.5 * fn.lam * sym ** 2 * 0.5 * grid.volume
    assert abs(tg["vw"] - ref) <= 1e-12 * ref
    # for a smooth field the two discrete forms differ by the discretisation error only: the
    # gap closes at the order of the scheme when the same field is sampled twice as finely
    gaps = []
    for n in (16, 32):
        u = W.random_field((n, n, n), seed=3, kind="smooth")
        g2 = O.Grid((n, n, n), (7.6, 7.6, 7.6), 6)
        zero = np.zeros(g2.shape)
        _, tl = O.ground_state_energy(u, zero, zero, g2, fn, 0.0, 0.0, 0.0)
        _, tg = O.ground_state_energy(u, zero, zero, g2, fn, 0.0, 0.0, 0.0, vw_energy="gradient")
        gaps.append(abs(tg["vw"] - tl["vw"]) / abs(tl["vw"]))
    assert gaps[0] < 1e-3 and gaps[1] < gaps[0] / 100, gaps


def test_ground_state_energy_and_forces_converge_at_order_2n():
    # Sec. 5.1: on the 4-atom cell with the corner atom moved to (0.80, 0.56, 0.42), the
    # errors of the ground-state energy and of the forces against a fine order-12 reference
    # fall as h^{2N} (measured rates between 16, 20 and 24 points per 7.6 bohr: energy 2.01 /
    # 3.9 / 5.7, forces 1.99 / 3.9 / 5.6 for N = 1 / 2 / 3).  A wrong weight, a dropped
    # stencil term or an energy term inconsistent with the Hamiltonian lowers the order.
    fn = O.tfw_functional()
    c = W.al4_displaced_cell(points_per_cell=16)
    g = O.Grid((40, 40, 40), c.L, 6)
    r = O.scf_ground_state(g, c.R, c.Z, c.sigma, c.rc, fn, nlcg_tol=1e-10)
    E_ref, F_ref = r.energy, O.forces(r.phi, c.R, c.Z, c.sigma, c.rc, g)
    ns = (16, 20, 24)
    for N in (1, 2, 3):
        e_err, f_err = [], []
        for n in ns:
            gn = O.Grid((n, n, n), c.L, N)
            rn = O.scf_ground_state(gn, c.R, c.Z, c.sigma, c.rc, fn, nlcg_tol=1e-10)
            e_err.append(abs(rn.energy - E_ref))
            f_err.append(np.abs(O.forces(rn.phi, c.R, c.Z, c.sigma, c.rc, gn) - F_ref).max())
        for errs in (e_err, f_err):
            rates = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(2)]
            assert min(rates) > 2 * N - 0.5, (N, errs, rates)


def test_preconditioned_nlcg_reaches_the_same_minimum_in_fewer_steps():
    # Sec. 5.5 asks for a real-space preconditioner for the NLCG: with the direction built from
    # (-L_h + shift)^{-1} r the method must end at the plain method's minimum (the line search
    # and the stopping test are unchanged) and get there in fewer steps
    cell = W.al4_lr_cell(points_per_cell=16)
    grid = O.Grid(cell.n, cell.L, 6)
    kw = dict(nlcg_tol=1e-8, fp_tol=1e-8, anderson_m=3, zeta=1.0)
    plain = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(), **kw)
    pre = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(),
                             precond_shift=8.0, **kw)
    assert abs(pre.energy - plain.energy) / cell.n_atoms < 1e-9
    assert np.max(np.abs(pre.u - plain.u)) < 1e-5 * np.max(plain.u)
    assert sum(pre.nlcg_iterations) < 0.6 * sum(plain.nlcg_iterations), (
        sum(pre.nlcg_iterations), sum(plain.nlcg_iterations))
    # the two-shift form (-L_h + 0.1)(-L_h + 1.2)^{-2}, which also follows the Hartree term's
    # 1/k^2 curvature at small k: the same minimum, fewer steps still (measured 59 against 86)
    two = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wt_functional(),
                             precond_shift=1.2, precond_low=0.1, **kw)
    assert abs(two.energy - plain.energy) / cell.n_atoms < 1e-9
    assert np.max(np.abs(two.u - plain.u)) < 1e-5 * np.max(plain.u)
    assert sum(two.nlcg_iterations) < 0.8 * sum(pre.nlcg_iterations), (
        sum(two.nlcg_iterations), sum(pre.nlcg_iterations))
    # the TFW functional (no outer loop) as well
    tcell = W.al4_displaced_cell(points_per_cell=16)
    tgrid = O.Grid(tcell.n, tcell.L, 6)
    tp = O.scf_ground_state(tgrid, tcell.R, tcell.Z, tcell.sigma, tcell.rc, O.tfw_functional(),
                            nlcg_tol=1e-8)
    tq = O.scf_ground_state(tgrid, tcell.R, tcell.Z, tcell.sigma, tcell.rc, O.tfw_functional(),
                            nlcg_tol=1e-8, precond_shift=8.0)
    assert abs(tq.energy - tp.energy) / tcell.n_atoms < 1e-9
    assert sum(tq.nlcg_iterations) < sum(tp.nlcg_iterations)
