"""Learned preconditioner for the shifted kernel systems through the C ABI.

The systems -(1/kf2) L_h W + Q W = P f of Sec. 3.1 are complex symmetric.  A network trained
(of_precond_set_shift) for the real positive operator -L_h + c, c = kf2 |Q| -- the operator
whose inverse the multigrid preconditioner of these systems approximates -- runs inside the
flexible CG of a few inner steps on that operator, applied to the real and imaginary parts of
each Arnoldi vector of flexible GMRES(8) (see oracle.precond.flexible_gmres).  Checked here: the
shifted loss and its gradients against the oracle network, the residuals collected from the real
shifted system, and the solve itself against the oracle's exact discrete solution, with what the
trained network gains over the same solver without it (every network step refused: plain inner
CG) and the fall-back when the network's directions are refused.

Tolerances as in test_gpu_precond.py (BF16 activations, FP32 sums); the solves are held to the
same 1e-9 relative bar as the other kernel-solve tests, since the stopping test uses the true
FP64 residual whatever the preconditioner.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import precond as NP  # noqa: E402
from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
H = 0.2375
GROUPS = ("W1", "b1", "W2", "b2", "W3", "b3")


def _bf16(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _flat(P):
    return np.concatenate([P[k].ravel() for k in GROUPS])


def _unflat(v, like):
    out, k0 = {}, 0
    for k in GROUPS:
        n = like[k].size
        out[k] = np.asarray(v[k0:k0 + n], dtype=np.float64).reshape(like[k].shape)
        k0 += n
    return out


def _wt_shift(k):
    """P and Q of the k-th conjugate pair of the WT-type kernel's rational fit (App. A)."""
    fn = Fn.wt()
    return complex(fn.P[4 * k], fn.P[4 * k + 1]), complex(fn.Q[4 * k], fn.Q[4 * k + 1])


def test_shifted_loss_and_gradients_match_oracle():
    n = (24, 20, 18)
    h = B.of_grid_create(n, tuple(H * m for m in n), 6, torch.cuda.current_stream())
    grid = O.Grid(n, tuple(H * m for m in n), 6)
    rng = np.random.default_rng(105)
    P = NP.init_params(seed=5)
    for k in ("b1", "b2", "b3"):
        P[k] = 0.1 * rng.normal(size=P[k].shape)
    P = {k: _bf16(v) for k, v in P.items()}
    c = 1.3
    try:
        net = B.of_precond_create(_flat(P))
        B.of_precond_set_shift(net, c)
        r = W.random_field(grid.shape, seed=11) + W.random_field(grid.shape, seed=12, kind="smooth")
        r = r.astype(np.float32).astype(np.float64)   # the shifted operator keeps the mean
        loss, g = B.of_precond_loss_grad(h, net, torch.tensor(r, dtype=torch.float32, device="cuda"))
        B.of_precond_destroy(net)
    finally:
        B.of_grid_destroy(h)
    ref_loss, ref = NP.loss_and_grads(P, r, grid, c)
    ref0, _ = NP.loss_and_grads(P, r, grid, 0.0)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
    assert abs(ref_loss - ref0) > 1e-2 * abs(ref0)   # the shift matters at this size
    G = _unflat(g, P)
    total = np.sqrt(sum(np.sum(ref[k] ** 2) for k in GROUPS))
    for k in GROUPS:
        e = np.linalg.norm(G[k] - ref[k])
        if k == "b3":
            assert e <= 5e-3 * total, (k, e, total)
        else:
            assert e <= 5e-3 * np.linalg.norm(ref[k]), (k, e / np.linalg.norm(ref[k]))


def _rhs(cell, kf2, seed=31):
    """A kernel-map right-hand side f = -(1/kf2) L_h g of a smooth positive field g (the form
    of Sec. 3.1's m = n = 0 right-hand side, with g standing in for u^{2 alpha})."""
    g = 1.0 + 0.5 * W.random_field(cell.shape, seed=seed, kind="smooth")
    grid = O.Grid(cell.n, cell.L, 6)
    return -O.laplacian(g, grid) / kf2, grid


def test_collect_residuals_of_a_shifted_system():
    cell = W.al4_cell()
    kf2 = Fn.kf2(cell.n_electrons, float(np.prod(cell.L)))
    f, _ = _rhs(cell, kf2)
    f = f + 0.3   # a mean the shifted system keeps
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        s = torch.zeros((10,) + cell.shape, dtype=torch.float32, device="cuda")
        cnt = B.of_precond_collect(h, torch.tensor(f, device="cuda"), 3, 10, s, shift=1.5)
        assert cnt == 10
        ref = f / np.sqrt(np.mean(f ** 2))   # the right-hand side at unit RMS, mean kept
        assert np.abs(s[0].double().cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
        rms = [float(torch.sqrt(torch.mean(s[k].double() ** 2))) for k in range(cnt)]
        assert rms[-1] < 0.5 * rms[0]
        with pytest.raises(B.OfError):
            B.of_precond_collect(h, torch.tensor(f, device="cuda"), 3, 10, s, shift=-1.0)
    finally:
        B.of_grid_destroy(h)


@pytest.fixture(scope="module")
def trained_shifted():
    """A network for the second WT shift (Q = 0.066 - 0.260i, c = kf2 |Q| = 0.93) on the
    108-atom 96^3 cell, trained (800 Adam steps) on every CG residual of the real system
    -L_h + c for four right-hand sides."""
    cell = W.al108_cell()
    kf2 = Fn.kf2(cell.n_electrons, float(np.prod(cell.L)))
    Pk, Qk = _wt_shift(1)
    c = kf2 * abs(Qk)
    net = B.of_precond_create(W.initial_network(4))
    B.of_precond_set_shift(net, c)
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    rng = np.random.default_rng(4)
    try:
        sets = []
        for seed in (41, 43, 45, 49):
            f, _ = _rhs(cell, kf2, seed)
            s = torch.empty((48,) + cell.shape, dtype=torch.float32, device="cuda")
            cnt = B.of_precond_collect(h, torch.tensor(f, device="cuda"), 1, 48, s, shift=c)
            sets += [s[k] for k in range(cnt)]
        S = torch.stack(sets).contiguous()
        cnt = S.shape[0]
        idx = np.linspace(0, cnt - 1, 16).astype(int)
        before = np.mean([B.of_precond_loss_grad(h, net, S[k])[0] for k in idx])
        for rnd in range(4):
            B.of_precond_train(h, net, S, cnt, rng.integers(0, cnt, size=800), 200, 4,
                               3e-3 if rnd < 3 else 1e-3)
        after = np.mean([B.of_precond_loss_grad(h, net, S[k])[0] for k in idx])
    finally:
        B.of_grid_destroy(h)
    yield net, (before, after), cell, kf2, Pk, Qk
    B.of_precond_destroy(net)


def _kernel_solve(cell, f, P, Q, kf2, opts):
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        Wc = torch.zeros(cell.shape + (2,), dtype=torch.float64, device="cuda")
        info = B.of_kernel_solve(h, torch.tensor(f, device="cuda"), [P], [Q], kf2, Wc, opts)
        w = Wc.cpu().numpy()
        return w[..., 0] + 1j * w[..., 1], info
    finally:
        B.of_grid_destroy(h)


def _opts(net=None, theta=0.3):
    o = B.of_default_solve_opts()
    o.tol = 1e-10
    o.precision = B.OF_F32
    o.no_multigrid = 1
    o.inner_tol = 1e-4
    if net is not None:
        o.precond = net
        o.precond_theta = theta
    return o


def test_training_on_shifted_residuals_lowers_the_loss(trained_shifted):
    _, (before, after), *_ = trained_shifted
    assert after < before and after < 0, (before, after)


def test_network_for_the_shift_cuts_gmres_iterations_same_answer(trained_shifted):
    net, _, cell, kf2, Pk, Qk = trained_shifted
    f, grid = _rhs(cell, kf2, seed=47)   # a right-hand side the network was not trained on
    ref = O.kernel_solve(f, grid, kf2, Pk, Qk)
    w_g, info_g = _kernel_solve(cell, f, Pk, Qk, kf2, _opts(net, theta=2.0))   # inner plain CG
    w_n, info_n = _kernel_solve(cell, f, Pk, Qk, kf2, _opts(net))              # with the net
    w_c, info_c = _kernel_solve(cell, f, Pk, Qk, kf2, _opts())                 # plain COCG
    scale = np.abs(ref).max()
    for w, info in ((w_g, info_g), (w_n, info_n), (w_c, info_c)):
        assert info.rel_residual <= 1e-10
        assert np.abs(w - ref).max() <= 1e-9 * scale
    assert info_g.net_steps == 0 and info_n.net_steps > 0
    # the network's gain: fewer iterations (outer GMRES plus inner CG) than the same solver
    # with plain inner CG, to the same true residual (measured 706 against 840 on a GB300; the
    # operator -L_h + c is well conditioned already, so the gain is modest)
    assert info_n.iterations < 0.92 * info_g.iterations, (info_n.iterations, info_g.iterations)


def test_refused_network_falls_back_to_plain_inner_cg(trained_shifted):
    # the negated network is never accepted: every inner step is the plain CG step, the same
    # arithmetic as with every network step refused by the threshold
    net, _, cell, kf2, Pk, Qk = trained_shifted
    p = B.of_precond_get_params(net).copy()
    k3 = 7809 - (16 * 27 + 1)
    p[k3:] *= -1.0
    bad = B.of_precond_create(p)
    try:
        f, grid = _rhs(cell, kf2, seed=47)
        _, info_g = _kernel_solve(cell, f, Pk, Qk, kf2, _opts(net, theta=2.0))
        w_b, info_b = _kernel_solve(cell, f, Pk, Qk, kf2, _opts(bad))
        assert info_b.net_steps == 0
        assert info_b.iterations == info_g.iterations, (info_b.iterations, info_g.iterations)
        ref = O.kernel_solve(f, grid, kf2, Pk, Qk)
        assert np.abs(w_b - ref).max() <= 1e-9 * np.abs(ref).max()
    finally:
        B.of_precond_destroy(bad)


def test_set_shift_rejects_a_negative_or_non_finite_shift():
    net = B.of_precond_create(_flat(NP.init_params(seed=1)))
    try:
        for bad in (-0.5, float("nan"), float("inf")):
            with pytest.raises(B.OfError):
                B.of_precond_set_shift(net, bad)
        B.of_precond_set_shift(net, 0.0)
    finally:
        B.of_precond_destroy(net)
