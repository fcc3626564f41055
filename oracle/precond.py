"""Learned preconditioner: a small 3D convolutional network and its training loss.

Oracle (test infrastructure only).  The paper suggests better preconditioning for its Krylov
solves (Sec. 5.5) without specifying one; this is the reference for the network used as a
preconditioner of the Poisson CG.  Network: three periodic 3x3x3 convolutions
1 -> 16 -> 16 -> 1 channels with biases, GELU (exact, erf form) after the first two.
Convolutions are cross-correlations, y[o](x) = b[o] + sum_c sum_t W[o][c][t] a[c](x + t),
t over the 27 offsets (dz, dy, dx) in {-1,0,1}^3 in that nesting order, indices periodic.

Loss for one residual r (normalised to unit RMS): the A-norm error of the correction y = net(r)
against the exact correction e = A^{-1} r, up to the constant 1/2 e^T A e:
    loss = 1/2 y^T A y - y^T r,   A = -L_h + c (Eq. FD:Laplacian),   d loss / d y = A y - r,
with c = 0 for the Poisson operator and c > 0 for a network that stands in for the inverse of
the real positive operator -L_h + c that approximates a shifted kernel system (Sec. 3.1,
-(1/kf2) L_h W + Q W = P f, scaled by kf2: c = kf2 |Q|).

The shifted systems are complex symmetric; flexible_gmres solves them by flexible GMRES(m)
preconditioned by a few steps of flexible CG with the network on -L_h + c, applied to the real
and imaginary parts of each Arnoldi vector separately.

Pins (tests/test_oracle_precond.py): every gradient against central finite differences of the
loss (c = 0 and c > 0); the periodic convolution against an explicit loop over offsets; the loss
against the A-norm error of the spectral solution (c = 0 and c > 0); the flexible CG against the
spectral solution without a preconditioner, in one step with the exact inverse, step for step
equal to CG when every network step is refused, and faster than CG with a linear SPD
preconditioner, and the shifted flexible CG against the spectral solution of -L_h + c; the
flexible GMRES against the minimal residual over the Krylov space (a dense least-squares solve
on a tiny grid), in one step with the exact inverse, and faster with the real positive
preconditioner, exact or by inner CG.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from .fd import Grid, laplacian

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
CHANNELS = 16


def init_params(seed=0, channels=CHANNELS):
    """He-style random initial weights (float64)."""
    rng = np.random.default_rng(seed)
    c = channels
    return dict(
        W1=rng.normal(0, np.sqrt(2.0 / 27), size=(c, 1, 27)), b1=np.zeros(c),
        W2=rng.normal(0, np.sqrt(2.0 / (27 * c)), size=(c, c, 27)), b2=np.zeros(c),
        W3=rng.normal(0, np.sqrt(1.0 / (27 * c)), size=(1, c, 27)), b3=np.zeros(1))


def shifted(a, t):
    """a(x + t) for an array of shape (..., n3, n2, n1), periodic."""
    dz, dy, dx = t
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(a, W, b):
    """Periodic 3x3x3 cross-correlation: a (C_in, n3, n2, n1) -> (C_out, n3, n2, n1)."""
    out = np.zeros((W.shape[0],) + a.shape[1:])
    for k, t in enumerate(OFFSETS):
        sa = shifted(a, t)
        out += np.einsum("oc,c...->o...", W[:, :, k], sa)
    return out + b[:, None, None, None]


def conv_backward(a, W, gy):
    """Gradients of sum(gy * conv(a, W, b)) with respect to W, b and a."""
    dW = np.zeros_like(W)
    ga = np.zeros_like(a)
    for k, t in enumerate(OFFSETS):
        sa = shifted(a, t)
        dW[:, :, k] = np.tensordot(gy, sa, axes=([1, 2, 3], [1, 2, 3]))
        # d/da: sum_x gy[o](x) W[o][c][t] a[c](x + t)  ->  ga[c](x') += W gy[o](x' - t)
        ga += np.einsum("oc,o...->c...", W[:, :, k], shifted(gy, tuple(-s for s in t)))
    db = gy.reshape(gy.shape[0], -1).sum(1)
    return dW, db, ga


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(P, r):
    """net(r) for r of shape (n3, n2, n1); returns (y, cache)."""
    a0 = r[None]
    z1 = conv(a0, P["W1"], P["b1"])
    a1 = gelu(z1)
    z2 = conv(a1, P["W2"], P["b2"])
    a2 = gelu(z2)
    y = conv(a2, P["W3"], P["b3"])[0]
    return y, (a0, z1, a1, z2, a2)


def loss_and_grads(P, r, grid: Grid, shift=0.0):
    """A-norm loss of one residual (r is normalised here to unit RMS) and its parameter
    gradients, A = -L_h + shift.  Returns (loss, grads dict)."""
    r = r / np.sqrt(np.mean(r * r))
    y, (a0, z1, a1, z2, a2) = forward(P, r)
    Ay = -laplacian(y, grid) + shift * y
    loss = 0.5 * float(np.sum(y * Ay)) - float(np.sum(y * r))
    gy = (Ay - r)[None]
    dW3, db3, ga2 = conv_backward(a2, P["W3"], gy)
    gz2 = ga2 * gelu_grad(z2)
    dW2, db2, ga1 = conv_backward(a1, P["W2"], gz2)
    gz1 = ga1 * gelu_grad(z1)
    dW1, db1, _ = conv_backward(a0, P["W1"], gz1)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3)


def apply(P, r):
    """Preconditioner z = s * net(r / s), s = RMS of r (homogeneous of degree one)."""
    s = np.sqrt(np.mean(r * r))
    if s == 0.0:
        return np.zeros_like(r)
    return s * forward(P, r / s)[0]


def flexible_cg(b, grid: Grid, P=None, tol=1e-8, theta=0.5, max_iter=5000, precond=None, m=4,
                shift=0.0):
    """Flexible CG on A x = b, A = -L_h + shift (truncated FCG(m) after Notay); for shift = 0
    (the Poisson operator) on mean-free fields.

    The preconditioned vector z (the network z = s net(r / s), or `precond(r)` when given, its
    mean removed when shift = 0) is kept only while it is a clear descent direction,
    cos(r, z) > theta; otherwise that iteration takes the plain direction z = r (Jacobi: the
    diagonal of A is a constant, so its inverse is a multiple of the identity, which the step
    length absorbs).  The direction is z made A-conjugate to the last m directions,
    p = z - sum_j (z^T A p_j / p_j^T A p_j) p_j, and the step is alpha = r^T p / p^T A p.
    Returns (x, iterations, network steps)."""
    def choose(r):
        if P is None and precond is None:
            return r.copy(), False
        z = precond(r) if precond is not None else apply(P, r)
        if shift == 0.0:
            z = z - z.mean()
        nz = np.linalg.norm(z)
        if nz > 0 and float(np.sum(r * z)) > theta * np.linalg.norm(r) * nz:
            return z, True
        return r.copy(), False

    x = np.zeros_like(b)
    r = b - b.mean() if shift == 0.0 else b.copy()
    nb = np.linalg.norm(r)
    if nb == 0.0:
        return x, 0, 0
    z, used = choose(r)
    net_steps = int(used)
    p = z
    past = []   # (p_j, A p_j, p_j^T A p_j), newest last
    for it in range(1, max_iter + 1):
        Ap = -laplacian(p, grid) + shift * p
        pAp = float(np.sum(p * Ap))
        alpha = float(np.sum(r * p)) / pAp
        x += alpha * p
        r = r - alpha * Ap
        past = (past + [(p, Ap, pAp)])[-m:]
        if np.linalg.norm(r) < tol * nb:
            return x, it, net_steps
        z, used = choose(r)
        net_steps += int(used)
        p = z.copy()
        for (pj, Apj, pApj) in past:
            p -= (float(np.sum(z * Apj)) / pApj) * pj
    return x, max_iter, net_steps


def flexible_gmres(f, grid: Grid, a, Q, P=None, tol=1e-8, m=8, max_iter=5000, precond=None,
                   inner=False, inner_tol=0.1, inner_max=40, theta=0.3):
    """Flexible GMRES(m) with right preconditioning (Saad's FGMRES) on the shifted system
    a (-L_h) x + Q x = f (the kernel systems of Sec. 3.1 with a = 1/kf2), complex.

    Preconditioner z_j = M(v_j): `precond(v_j)` when given; with inner=True, flexible CG with
    the network P (plain CG when P is None) on the real positive operator -L_h + c, c = |Q| / a,
    applied to the real and imaginary parts of v_j separately and stopped at relative residual
    inner_tol (or after inner_max steps); otherwise z_j = v_j (GMRES).  The system is complex
    symmetric, not Hermitian, and M is neither linear nor complex-homogeneous, so no short
    recurrence stays valid: FGMRES keeps every z_j of a cycle and takes the iterate that
    minimises the residual over their span.  w = A z_j orthogonalised against v_0..v_j by
    modified Gram-Schmidt (Hermitian products) gives column j of the Hessenberg matrix H and
    v_{j+1}; min_y |beta e_1 - H y| is the residual of x_0 + Z y.  After m steps, or once that
    residual is below tol |f|, x takes the minimiser and the cycle restarts from the true
    residual.  Returns (x, outer iterations, inner iterations, network steps)."""
    def A(v):
        return -a * (laplacian(v.real, grid) + 1j * laplacian(v.imag, grid)) + Q * v

    c = abs(Q) / a
    counts = [0, 0]   # inner iterations, network steps

    def M(v):
        if precond is not None:
            return precond(v)
        if not inner:
            return v.copy()
        parts = []
        for part in (v.real, v.imag):
            zp, its, used = flexible_cg(part, grid, P=P, tol=inner_tol, theta=theta,
                                        max_iter=inner_max, shift=c)
            counts[0] += its
            counts[1] += used
            parts.append(zp)
        return parts[0] + 1j * parts[1]

    f = np.asarray(f, dtype=complex)
    x = np.zeros_like(f)
    nb = np.linalg.norm(f)
    if nb == 0.0:
        return x, 0, 0, 0
    r = f.copy()
    it = 0
    while it < max_iter:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=complex)
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            k = j + 1
            e1 = np.zeros(k + 1, dtype=complex)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            est = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
            if est < tol * nb or H[j + 1, j] == 0.0 or it >= max_iter:
                break
            V.append(w / H[j + 1, j])
        x = x + sum(yi * zi for yi, zi in zip(y, Z))
        r = f - A(x)
        if np.linalg.norm(r) < tol * nb:
            break
    return x, it, counts[0], counts[1]
