"""Pins of the oracle's learned-preconditioner network: convolution, gradients, and the
effect of a trained network on CG iterations."""
import numpy as np
import pytest

import oracle as O
from oracle import precond as NP
from paper_1412_8250_gb300 import workloads as W


def test_conv_matches_explicit_offsets():
    rng = np.random.default_rng(0)
    a = rng.normal(size=(2, 5, 6, 7))
    Wt = rng.normal(size=(3, 2, 27))
    b = rng.normal(size=3)
    y = NP.conv(a, Wt, b)
    n3, n2, n1 = a.shape[1:]
    for (o, z, yy, x) in [(0, 0, 0, 0), (2, 4, 5, 6), (1, 2, 3, 1)]:
        s = b[o]
        for c in range(2):
            for k, (dz, dy, dx) in enumerate(NP.OFFSETS):
                s += Wt[o, c, k] * a[c, (z + dz) % n3, (yy + dy) % n2, (x + dx) % n1]
        assert abs(y[o, z, yy, x] - s) < 1e-12


@pytest.mark.parametrize("shift", [0.0, 1.7])
def test_gradients_match_finite_differences(shift):
    grid = O.Grid((6, 7, 8), (1.5, 1.7, 1.9), 3)
    P = NP.init_params(seed=1, channels=4)
    for k in P:
        P[k] = P[k] + 0.05 * np.random.default_rng(3).normal(size=P[k].shape)
    r = W.random_field(grid.shape, seed=5)
    loss, G = NP.loss_and_grads(P, r, grid, shift)
    rng = np.random.default_rng(9)
    e = 1e-6
    for name in P:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += e
            Pm[name][idx] -= e
            fd = (NP.loss_and_grads(Pp, r, grid, shift)[0] - NP.loss_and_grads(Pm, r, grid, shift)[0]) / (2 * e)
            assert abs(fd - G[name][idx]) < 1e-5 * max(1.0, abs(fd)), (name, idx)


def test_loss_is_a_norm_error_up_to_a_constant():
    # 1/2 y^T A y - y^T r + 1/2 e^T A e = 1/2 (y - e)^T A (y - e) with A e = r
    grid = O.Grid((8, 8, 8), (2.0, 2.0, 2.0), 6)
    P = NP.init_params(seed=2, channels=4)
    r = W.random_field(grid.shape, seed=6)
    r -= r.mean()
    loss, _ = NP.loss_and_grads(P, r, grid)
    rn = r / np.sqrt(np.mean(r * r))
    e = O.solve_shifted_spectral(rn, grid, 1.0, 0.0)
    y, _ = NP.forward(P, rn)
    d = y - e
    d -= d.mean()
    lhs = loss + 0.5 * float(np.sum(e * -O.laplacian(e, grid)))
    rhs = 0.5 * float(np.sum(d * -O.laplacian(d, grid)))
    # the constant mode of y is invisible to A; the y^T r term sees it only through mean(r) = 0
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(rhs))


def _poisson_case(n=12, seed=11):
    grid = O.Grid((n, n, n), (0.2375 * n,) * 3, 6)
    b = W.random_field(grid.shape, seed=seed, kind="smooth") + 0.3 * W.random_field(grid.shape, seed=seed + 1)
    b -= b.mean()
    return grid, b, O.solve_shifted_spectral(b, grid, 1.0, 0.0)


def test_flexible_cg_without_preconditioner_is_cg():
    # no preconditioner: every step is the plain CG step; the answer is the spectral solution
    grid, b, x_exact = _poisson_case()
    x, its, used = NP.flexible_cg(b, grid, tol=1e-10)
    x -= x.mean()
    assert used == 0 and 5 < its < 500
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)


def test_flexible_cg_with_exact_inverse_takes_one_step():
    # M = A^{-1}: the first direction is the exact correction
    grid, b, x_exact = _poisson_case()
    inv = lambda r: O.solve_shifted_spectral(r - r.mean(), grid, 1.0, 0.0)  # noqa: E731
    x, its, used = NP.flexible_cg(b, grid, tol=1e-10, precond=inv)
    assert its == 1 and used == 1


def test_flexible_cg_falls_back_on_an_ascent_direction():
    # M r = -r is never accepted: the iteration is the plain one step for step
    grid, b, _ = _poisson_case()
    _, its_plain, _ = NP.flexible_cg(b, grid, tol=1e-10)
    _, its, used = NP.flexible_cg(b, grid, tol=1e-10, precond=lambda r: -r)
    assert used == 0 and its == its_plain


def test_flexible_cg_with_spd_preconditioner_beats_cg():
    # a linear SPD preconditioner (inverse of A + c) is accepted at every step with theta = 0
    # and needs fewer iterations than CG; the answer is unchanged
    grid, b, x_exact = _poisson_case()
    M = lambda r: O.solve_shifted_spectral(r, grid, 1.0, 2.0)  # noqa: E731
    _, its_plain, _ = NP.flexible_cg(b, grid, tol=1e-10)
    x, its, used = NP.flexible_cg(b, grid, tol=1e-10, theta=0.0, precond=M)
    x -= x.mean()
    assert used == its and its < its_plain
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)


def test_flexible_cg_keeps_conjugacy_with_more_directions():
    # with a linear SPD preconditioner, orthogonalising against more past directions changes
    # nothing in exact arithmetic (PCG directions are already A-conjugate): same count
    grid, b, _ = _poisson_case()
    M = lambda r: O.solve_shifted_spectral(r, grid, 1.0, 2.0)  # noqa: E731
    counts = [NP.flexible_cg(b, grid, tol=1e-10, theta=0.0, precond=M, m=m)[1] for m in (1, 4, 8)]
    assert max(counts) - min(counts) <= 1, counts


def test_shifted_loss_is_a_norm_error_up_to_a_constant():
    # A = -L_h + c is positive definite: 1/2 y^T A y - y^T r + 1/2 e^T A e = 1/2 (y-e)^T A (y-e)
    grid = O.Grid((8, 8, 8), (2.0, 2.0, 2.0), 6)
    c = 2.5
    P = NP.init_params(seed=2, channels=4)
    r = W.random_field(grid.shape, seed=6)
    loss, _ = NP.loss_and_grads(P, r, grid, c)
    rn = r / np.sqrt(np.mean(r * r))
    e = O.solve_shifted_spectral(rn, grid, 1.0, c)
    y, _ = NP.forward(P, rn)
    d = y - e
    A = lambda v: -O.laplacian(v, grid) + c * v  # noqa: E731
    lhs = loss + 0.5 * float(np.sum(e * A(e)))
    rhs = 0.5 * float(np.sum(d * A(d)))
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(rhs))


A_SC, Q_SH = 1.0 / 3.5, 0.3 + 0.5j   # a = 1/kf2 of an aluminium-like density, a complex shift


def _shifted_case(n=12, seed=21):
    grid = O.Grid((n, n, n), (0.2375 * n,) * 3, 6)
    f = W.random_field(grid.shape, seed=seed, kind="smooth") + 0.3 * W.random_field(grid.shape, seed=seed + 1)
    return grid, f, O.solve_shifted_spectral(f.astype(complex), grid, A_SC, Q_SH)


def _dense_operator(grid):
    """A = a (-L_h) + Q as a dense matrix, column k = A e_k (flattened in numpy order)."""
    n = int(np.prod(grid.shape))
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(-A_SC * O.laplacian(e.reshape(grid.shape), grid).ravel() + Q_SH * e)
    return np.array(cols).T


def test_flexible_gmres_without_preconditioner_minimises_the_residual():
    # k unpreconditioned steps from x = 0 reach the smallest residual over the Krylov space
    # span{f, A f, ..., A^{k-1} f}: a dense least-squares solve with an orthonormal basis of it
    grid = O.Grid((5, 5, 5), (1.3, 1.4, 1.5), 1)
    rng = np.random.default_rng(4)
    f = rng.normal(size=grid.shape) + 1j * rng.normal(size=grid.shape)
    Ad = _dense_operator(grid)
    fv = f.ravel()
    K = [fv]
    for k in range(1, 7):
        x, its, _, _ = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-14, m=10, max_iter=k)
        assert its == k
        Qk, _ = np.linalg.qr(np.array(K).T)
        y = np.linalg.lstsq(Ad @ Qk, fv, rcond=None)[0]
        best = np.linalg.norm(fv - Ad @ (Qk @ y))
        got = np.linalg.norm(fv - Ad @ x.ravel())
        assert abs(got - best) <= 1e-9 * np.linalg.norm(fv), (k, got, best)
        K.append(Ad @ K[-1])


def test_flexible_gmres_converges_to_the_spectral_solution():
    grid, f, x_exact = _shifted_case()
    x, its, inner, used = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-10, m=8)
    assert inner == 0 and used == 0 and 5 < its < 2000
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)


def test_flexible_gmres_with_exact_inverse_takes_one_step():
    grid, f, x_exact = _shifted_case()
    inv = lambda v: O.solve_shifted_spectral(v, grid, A_SC, Q_SH)  # noqa: E731
    x, its, _, _ = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-10, precond=inv)
    assert its == 1
    assert np.linalg.norm(x - x_exact) <= 1e-10 * np.linalg.norm(x_exact)


def test_shifted_flexible_cg_solves_the_real_positive_operator():
    # A = -L_h + c keeps the constant mode: no projection, the spectral solution of -L_h + c
    grid, f, _ = _shifted_case()
    c = abs(Q_SH) / A_SC
    x, its, used = NP.flexible_cg(f, grid, tol=1e-11, shift=c)
    ref = O.solve_shifted_spectral(f, grid, 1.0, c)
    assert used == 0 and its > 3
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # with a linear SPD preconditioner accepted at every step, fewer steps, the same answer
    M = lambda r: O.solve_shifted_spectral(r, grid, 1.0, 2.0 * c)  # noqa: E731
    x2, its2, used2 = NP.flexible_cg(f, grid, tol=1e-11, theta=0.0, precond=M, shift=c)
    assert used2 == its2 and its2 < its
    assert np.linalg.norm(x2 - ref) <= 1e-9 * np.linalg.norm(ref)


def test_flexible_gmres_with_the_real_positive_preconditioner_beats_gmres():
    # the real operator -L_h + kf2 |Q| inverted on real and imaginary parts -- exactly, or by
    # inner CG to 1e-1 -- the preconditioner the network stands in for (and the one the
    # multigrid V-cycle approximates)
    grid, f, x_exact = _shifted_case()
    c = abs(Q_SH) / A_SC
    M = lambda v: O.solve_shifted_spectral(v, grid, 1.0, c)  # noqa: E731
    _, its_plain, _, _ = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-10, m=8)
    x, its, _, _ = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-10, m=8, precond=M)
    assert its < its_plain / 2
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)
    x, its_in, inner, used = NP.flexible_gmres(f, grid, A_SC, Q_SH, tol=1e-10, m=8, inner=True)
    assert used == 0 and inner > its_in and its_in < its_plain / 2
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)
