"""Electronic ground state: Hamiltonian, energies, the constrained NLCG of App. C, Anderson
mixing of App. D and the fixed point on V_LR of Sec. 3.3.1 (arXiv:1412.8250).

Oracle (test infrastructure only).  Readings used:
  * vW energy as -(lam/2) int u L_h u (so that dE/du = 2 dV H u holds exactly on the grid);
  * inner products <a, b> = dV sum a b, norm ||a|| = sqrt(<a, a>);
  * NLCG moves along the conjugate direction d_q (the printed update uses r_q, which would
    leave d_q unused); s ranges over the reals, so the sign is absorbed;
  * the loop stops as soon as ||r_q|| / sqrt(N_e) < tol, before a line search;
  * restart (d_q = r_q) at q = 0, every N_restart steps and whenever xi <= 0;
  * the line-search energy E(s) is evaluated exactly: phi(s) follows from phi(0) by
    linearity of the Poisson problem, phi(s) = c^2 (phi_uu + 2 s phi_ud + s^2 phi_dd) + phi_b
    with c = sqrt(N_e)/||u + s d||, so no Poisson solve is needed per trial s;
  * Anderson: m columns of history, zeta the mixing parameter, first step V_1 = V_0 + zeta f_0;
    fixed-point error ||f_k|| / ||V^hat_k||;
  * for mu = 0 (TFW) the inner minimisation is the ground state and the outer loop is skipped.

Pins (tests/test_oracle_scf.py): dE/du = 2 dV H u by central differences; the NLCG minimum
equals the minimum found by an independent L-BFGS minimisation; the Euler-Lagrange residual
and the constraint at convergence; Anderson with zeta = 1 and unbounded history equals the
GMRES-based iterate g(x_k^GMRES) on a linear fixed point (Walker & Ni); the line-search
energy via linearity equals a fresh Poisson solve.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import pi, sqrt

import numpy as np
from scipy.optimize import brent

from .fd import Grid, gradient, laplacian, integrate, poisson_solve, solve_shifted_spectral
from .functional import tf_energy_density, tf_potential, xc_energy_density, v_xc
from .kernel import Functional, lr_potential, kf2_of
from .pseudo import pseudocharge, self_energy, repulsive_correction


def inner(a, b, grid: Grid) -> float:
    return float(grid.dV * np.sum(a * b))


def hamiltonian_apply(u, phi, V_LR, grid: Grid, fn: Functional):
    """H u with H = -(lam/2) lap + V_TF + mu V_LR + V_xc + phi (Eq. EulerLagrange)."""
    rho = u * u
    V = tf_potential(rho) + v_xc(rho) + phi
    if fn.mu != 0.0:
        V = V + fn.mu * V_LR
    return -0.5 * fn.lam * laplacian(u, grid) + V * u


def inner_energy(u, phi, b, V_LR, grid: Grid, fn: Functional) -> float:
    """The functional of Eq. MVF at fixed V_LR, evaluated at its electrostatic supremum
    (value 1/2 int (u^2 + b) phi with phi the Poisson solution), without the constant
    self-energy and overlap terms."""
    rho = u * u
    e = (tf_energy_density(rho) - 0.5 * fn.lam * u * laplacian(u, grid)
         + xc_energy_density(rho) + 0.5 * (rho + b) * phi)
    if fn.mu != 0.0:
        e = e + fn.mu * V_LR * rho
    return integrate(e, grid)


GOLD = 1.618033988749895


def line_minimum(f, s_try, max_expand=60, max_shrink=60):
    """Brent's method (Sec. 4; scipy's implementation) on a bracket found from s = 0 along
    increasing s: expand by the golden ratio while f decreases, shrink the trial step while
    it does not.  Returns 0.0 when no decrease is found (f flat to rounding)."""
    f0 = f(0.0)
    b = abs(s_try)
    fb = f(b)
    if fb < f0:
        a, fa = 0.0, f0
        c = b * (1.0 + GOLD)
        fc = f(c)
        k = 0
        while fc < fb and k < max_expand:
            a, fa, b, fb = b, fb, c, fc
            c = b + GOLD * (b - a)
            fc = f(c)
            k += 1
        if fc < fb:
            return c
        if not fc > fb:                     # flat to rounding between b and c
            return b
    else:
        c, fc = b, fb
        b = c / (1.0 + GOLD)
        fb = f(b)
        k = 0
        while fb >= f0 and k < max_shrink:
            c, fc = b, fb
            b = c / (1.0 + GOLD)
            fb = f(b)
            k += 1
        if fb >= f0:
            return 0.0
        a, fa = 0.0, f0
    return float(brent(f, brack=(a, b, c), tol=1e-8))


@dataclass
class NlcgInfo:
    iterations: int = 0
    residual: float = float("inf")
    converged: bool = False
    steps: list = field(default_factory=list)


def nlcg(u0, V_LR, b, phi_b, grid: Grid, fn: Functional, n_electrons, tol=1e-6,
         max_iter=2000, n_restart=50, s_init=1e-2, precond_shift=0.0, precond_low=0.0):
    """Constrained non-linear CG with Polak-Ribiere update and Brent line search (App. C,
    Algorithm NLCG).  Returns (u, phi, info) with phi the Poisson solution for u.

    precond_shift > 0: the real-space preconditioner for the NLCG that Sec. 5.5 calls for, in
    its plainest form: the direction is built from z = (-L_h + precond_shift)^{-1} r (solved
    exactly here) with the preconditioned Polak-Ribiere coefficient
    xi = <z, r - r_prev> / <z_prev, r_prev>; the line search and the stopping test are those of
    the plain method, so the minimum reached is the same.

    precond_low > 0 as well: z = (-L_h + precond_low) (-L_h + precond_shift)^{-2} r.  The
    energy's curvature along a density wave of wave number k grows like k^2 at large k (the vW
    term) and like 16 pi rho_bar / k^2 at small k (the Hartree term, which a larger cell reaches
    with smaller k); this form decays like 1/k^2 at large k and flattens at small k, so that it
    follows both ends."""
    Ne = float(n_electrons)
    u = u0 * sqrt(Ne / inner(u0, u0, grid))
    phi = poisson_solve(u * u + b, grid)
    info = NlcgInfo()
    r_prev = d_prev = z_prev = None
    s_prev = s_init
    for q in range(max_iter + 1):
        Hu = hamiltonian_apply(u, phi, V_LR, grid, fn)
        eta = inner(u, Hu, grid) / Ne
        r = -2.0 * (Hu - eta * u)
        info.residual = sqrt(inner(r, r, grid)) / sqrt(Ne)
        info.iterations = q
        if info.residual < tol:
            info.converged = True
            break
        if q == max_iter:
            break
        if precond_shift > 0.0 and precond_low > 0.0:
            t = solve_shifted_spectral(solve_shifted_spectral(r, grid, 1.0, precond_shift).real,
                                       grid, 1.0, precond_shift).real
            z = -laplacian(t, grid) + precond_low * t
        elif precond_shift > 0.0:
            z = solve_shifted_spectral(r, grid, 1.0, precond_shift).real
        else:
            z = r
        if q == 0 or q % n_restart == 0:
            d = z
        else:
            xi = inner(r - r_prev, z, grid) / inner(r_prev, z_prev, grid)
            d = z if xi <= 0.0 else z + xi * d_prev
        phi_uu = phi - phi_b
        phi_ud = poisson_solve(u * d, grid)
        phi_dd = poisson_solve(d * d, grid)

        def energy_at(s):
            w = u + s * d
            c2 = Ne / inner(w, w, grid)
            us = sqrt(c2) * w
            phis = c2 * (phi_uu + 2.0 * s * phi_ud + s * s * phi_dd) + phi_b
            return inner_energy(us, phis, b, V_LR, grid, fn)

        slope = -inner(r, d, grid)          # dE/ds at s = 0 for the normalised path
        if slope >= 0.0:                    # not a descent direction: restart along r
            d = r
            phi_ud = poisson_solve(u * d, grid)
            phi_dd = poisson_solve(d * d, grid)
        s = line_minimum(energy_at, s_prev)
        if s == 0.0:                        # energy flat to rounding along d: stagnated
            info.steps.append(0.0)
            break
        w = u + s * d
        u = sqrt(Ne / inner(w, w, grid)) * w
        phi = poisson_solve(u * u + b, grid)
        info.steps.append(s)
        r_prev, d_prev, z_prev = r, d, z
        s_prev = s if s != 0.0 else s_init
    return u, phi, info


def anderson_update(V_hist, f_hist, zeta, m):
    """App. D: V_{k+1} = V_k + zeta f_k - (S_k + zeta Y_k)(Y_k^T Y_k)^{-1} Y_k^T f_k, with
    S_k, Y_k the last m differences of iterates and residuals.  The normal-equation product
    (Y^T Y)^{-1} Y^T f is taken as the least-squares solution of Y gamma = f."""
    Vk, fk = V_hist[-1], f_hist[-1]
    k = len(V_hist) - 1
    j = min(m, k)
    if j == 0:
        return Vk + zeta * fk
    cols = range(k - j + 1, k + 1)
    S = np.stack([(V_hist[i] - V_hist[i - 1]).ravel() for i in cols], axis=1)
    Y = np.stack([(f_hist[i] - f_hist[i - 1]).ravel() for i in cols], axis=1)
    gamma = np.linalg.lstsq(Y, fk.ravel(), rcond=None)[0]
    return Vk + zeta * fk - ((S + zeta * Y) @ gamma).reshape(Vk.shape)


@dataclass
class ScfResult:
    u: np.ndarray
    phi: np.ndarray
    V_LR: np.ndarray
    energy: float
    terms: dict
    outer_iterations: int
    nlcg_iterations: list
    fp_errors: list


def ground_state_energy(u, phi, b, grid: Grid, fn: Functional, T_LR, E_self, E_c,
                        vw_energy="laplacian"):
    """Eq. GroundStateEnergy: TF + lam vW + mu T_LR + xc + 1/2 int (u^2 + b) phi
    - 1/2 sum_J int b_J V_J + E_c^*.  The vW term is -(lam/2) int u L_h u (the discrete form
    whose gradient is the Hamiltonian, R7) or, with vw_energy="gradient", (lam/2) int |grad_h u|^2
    with the order-2N gradient of Eq. gradient:approximate (Eq. vW:KineticEnergy as printed)."""
    rho = u * u
    if vw_energy == "gradient":
        vw = integrate(0.5 * fn.lam * np.sum(gradient(u, grid) ** 2, axis=0), grid)
    else:
        vw = integrate(-0.5 * fn.lam * u * laplacian(u, grid), grid)
    t = dict(
        tf=integrate(tf_energy_density(rho), grid),
        vw=vw,
        lr=fn.mu * T_LR,
        xc=integrate(xc_energy_density(rho), grid),
        es=integrate(0.5 * (rho + b) * phi, grid),
        self=E_self,
        corr=E_c,
    )
    return float(sum(t.values())), t


def scf_ground_state(grid: Grid, R, Z, sigma, rc, fn: Functional, u0=None, nlcg_tol=1e-7,
                     fp_tol=1e-7, max_outer=50, anderson_m=7, zeta=0.3, n_restart=50,
                     max_nlcg=5000, fixed_point="V", vw_energy="laplacian", precond_shift=0.0,
                     precond_low=0.0):
    """Fixed point V_LR = V[U(V_LR)] (Eqs. FixedPoint:Map1, MVF) with Anderson mixing
    (App. D); V_LR,0 = 0.  Returns the ground state and its energy.

    fixed_point="u": the alternative the paper compares in Sec. 5.3 (Table MixComparison), the
    fixed point u = U(V[u]) with Anderson mixing of u (renormalised to N_e before each map),
    error ||U(V[u_k]) - u_k|| / ||U(V[u_k])||, the energy taken at u = U(V[u_k])."""
    if fixed_point == "u" and fn.mu != 0.0:
        return _scf_ground_state_u(grid, R, Z, sigma, rc, fn, u0, nlcg_tol, fp_tol, max_outer,
                                   anderson_m, zeta, n_restart, max_nlcg, vw_energy)
    Ne = float(np.sum(Z))
    b = pseudocharge(R, Z, sigma, rc, grid)
    phi_b = poisson_solve(b, grid)
    E_self = self_energy(R, Z, sigma, rc, grid)
    E_c = repulsive_correction(R, Z, sigma, grid.L)
    kf2 = kf2_of(Ne, grid.volume)
    u = np.full(grid.shape, sqrt(Ne / grid.volume)) if u0 is None else u0.copy()
    V = np.zeros(grid.shape)
    V_hist, f_hist, errs, its = [], [], [], []
    T_LR = 0.0
    for k in range(max_outer):
        u, phi, info = nlcg(u, V, b, phi_b, grid, fn, Ne, tol=nlcg_tol, max_iter=max_nlcg,
                            n_restart=n_restart, precond_shift=precond_shift,
                            precond_low=precond_low)
        its.append(info.iterations)
        if fn.mu == 0.0:
            break
        Vhat, T_LR, _, _ = lr_potential(u, grid, fn, kf2)
        f = Vhat - V
        errs.append(float(np.linalg.norm(f) / np.linalg.norm(Vhat)))
        V_hist.append(V)
        f_hist.append(f)
        if errs[-1] < fp_tol:
            break
        V = anderson_update(V_hist, f_hist, zeta, anderson_m)
    E, terms = ground_state_energy(u, phi, b, grid, fn, T_LR, E_self, E_c, vw_energy)
    return ScfResult(u=u, phi=phi, V_LR=V, energy=E, terms=terms, outer_iterations=len(its),
                     nlcg_iterations=its, fp_errors=errs)


def _scf_ground_state_u(grid, R, Z, sigma, rc, fn, u0, nlcg_tol, fp_tol, max_outer, anderson_m,
                        zeta, n_restart, max_nlcg, vw_energy):
    Ne = float(np.sum(Z))
    b = pseudocharge(R, Z, sigma, rc, grid)
    phi_b = poisson_solve(b, grid)
    E_self = self_energy(R, Z, sigma, rc, grid)
    E_c = repulsive_correction(R, Z, sigma, grid.L)
    kf2 = kf2_of(Ne, grid.volume)
    x = np.full(grid.shape, sqrt(Ne / grid.volume)) if u0 is None else u0.copy()
    x_hist, f_hist, errs, its = [], [], [], []
    for k in range(max_outer):
        x = x * sqrt(Ne / inner(x, x, grid))
        V, _, _, _ = lr_potential(x, grid, fn, kf2)
        u, phi, info = nlcg(x, V, b, phi_b, grid, fn, Ne, tol=nlcg_tol, max_iter=max_nlcg,
                            n_restart=n_restart)
        its.append(info.iterations)
        f = u - x
        errs.append(float(np.linalg.norm(f) / np.linalg.norm(u)))
        x_hist.append(x)
        f_hist.append(f)
        if errs[-1] < fp_tol:
            break
        x = anderson_update(x_hist, f_hist, zeta, anderson_m)
    V_u, T_LR, _, _ = lr_potential(u, grid, fn, kf2)
    E, terms = ground_state_energy(u, phi, b, grid, fn, T_LR, E_self, E_c, vw_energy)
    return ScfResult(u=u, phi=phi, V_LR=V_u, energy=E, terms=terms, outer_iterations=len(its),
                     nlcg_iterations=its, fp_errors=errs)
