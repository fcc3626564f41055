"""Learned preconditioner through the C ABI: network and gradients against the oracle network,
training on the GPU, and what the trained network gains in the Poisson solve.

Tolerances.  The kernels keep the weights, the scaled input r / s and the activations z1, a1,
z2, a2 in BF16 (relative rounding <= 2^-9) and sum in FP32.  The oracle runs in FP64 on the same
BF16-rounded weights.  Repeating the oracle with its input and activations rounded to BF16
gives, on these inputs, an RMS error of 0.37 % in the output, 0.012 % in the loss and <= 0.1 %
in each weight gradient; the bars below are four to five times those.  db3 = sum(A y - r) is close to zero, so
its bar is absolute, relative to the size of the whole gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import precond as NP  # noqa: E402
from paper_1412_8250_gb300 import binding as B, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
H = 0.2375   # grid spacing of the aluminium cells (a = 7.6 bohr, 32 points per cell)
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


def _params(seed):
    P = NP.init_params(seed=seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        P[k] = 0.1 * rng.normal(size=P[k].shape)
    return {k: _bf16(v) for k, v in P.items()}


def _grid(n):
    h = B.of_grid_create(n, tuple(H * m for m in n), 6, torch.cuda.current_stream())
    return h, O.Grid(n, tuple(H * m for m in n), 6)


def _field(shape, seed):
    r = W.random_field(shape, seed=seed) + W.random_field(shape, seed=seed + 1, kind="smooth")
    return (r - r.mean()).astype(np.float32).astype(np.float64)


def test_parameter_count():
    assert B.of_precond_num_params() == _flat(NP.init_params()).size == 7809


def test_forward_matches_oracle_network():
    n = (28, 24, 20)   # n1, n2, n3: 13440 points, a ragged last block of 256
    h, grid = _grid(n)
    P = _params(3)
    try:
        net = B.of_precond_create(_flat(P))
        r = _field(grid.shape, 7)
        rd = torch.tensor(r, dtype=torch.float32, device="cuda")
        z = torch.empty_like(rd)
        B.of_precond_apply(h, net, rd, z)
        ref = NP.apply(P, r)
        got = z.cpu().numpy().astype(np.float64)
        err = got - ref
        assert np.sqrt(np.mean(err ** 2)) <= 1.5e-2 * np.sqrt(np.mean(ref ** 2))
        assert np.abs(err).max() <= 2e-2 * np.abs(ref).max()
        # homogeneous of degree one: z(c r) = c z(r)
        B.of_precond_apply(h, net, rd * 4.0, z)
        assert np.abs(z.cpu().numpy() - 4.0 * got).max() <= 1e-5 * np.abs(got).max() * 4.0
        B.of_precond_destroy(net)
    finally:
        B.of_grid_destroy(h)


def test_loss_and_gradients_match_oracle():
    n = (24, 20, 18)
    h, grid = _grid(n)
    P = _params(5)
    try:
        net = B.of_precond_create(_flat(P))
        r = _field(grid.shape, 11)
        loss, g = B.of_precond_loss_grad(h, net, torch.tensor(r, dtype=torch.float32, device="cuda"))
        B.of_precond_destroy(net)
    finally:
        B.of_grid_destroy(h)
    ref_loss, ref = NP.loss_and_grads(P, r, grid)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
    G = _unflat(g, P)
    total = np.sqrt(sum(np.sum(ref[k] ** 2) for k in GROUPS))
    for k in GROUPS:
        e = np.linalg.norm(G[k] - ref[k])
        if k == "b3":
            assert e <= 5e-3 * total, (k, e, total)
        else:
            assert e <= 5e-3 * np.linalg.norm(ref[k]), (k, e / np.linalg.norm(ref[k]))


def _density(cell, n):
    """Uniform electron density plus the ions' pseudocharges: the right-hand side of the first
    Poisson solve of a ground-state run on that cell."""
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        b = torch.zeros(cell.shape, dtype=torch.float64, device="cuda")
        B.of_pseudocharge(h, B.make_system(cell.R, cell.Z, cell.sigma, cell.rc), b)
        omega = float(np.prod(cell.L))
        return b + cell.n_electrons / omega
    finally:
        B.of_grid_destroy(h)


def _mean_loss(h, net, samples, idx):
    return float(np.mean([B.of_precond_loss_grad(h, net, samples[k])[0] for k in idx]))


def _train(cells, strides, steps=400, batch=4, lr=3e-3, seed=0):
    """Collects CG residuals of each cell's Poisson solve and trains a fresh network on them,
    alternating between the cells in four Adam runs each (the last at lr / 3).  Returns the
    network and, per cell, the mean loss of eight fixed samples before and after training."""
    P0 = {k: 0.3 * v for k, v in NP.init_params(seed=seed).items()}
    net = B.of_precond_create(_flat(P0))
    data = []
    rng = np.random.default_rng(seed)
    try:
        for cell, stride in zip(cells, strides):
            rho = _density(cell, cell.n)
            h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
            data.append([h, None, 0])
            samples = torch.empty((64,) + cell.shape, dtype=torch.float32, device="cuda")
            data[-1][1:] = [samples, B.of_precond_collect(h, rho, stride, 64, samples)]
        evals = [np.linspace(0, cnt - 1, 8).astype(int) for (_, _, cnt) in data]
        before = [_mean_loss(h, net, s, e) for (h, s, _), e in zip(data, evals)]
        for rnd in range(4):
            for (h, samples, cnt) in data:
                st = steps // 4
                order = rng.integers(0, cnt, size=st * batch)
                B.of_precond_train(h, net, samples, cnt, order, st, batch, lr if rnd < 3 else lr / 3)
        after = [_mean_loss(h, net, s, e) for (h, s, _), e in zip(data, evals)]
    finally:
        for (h, _, _) in data:
            B.of_grid_destroy(h)
    return net, list(zip(before, after))


def test_collect_residuals():
    cell = W.al4_cell()
    rho = _density(cell, cell.n)
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        s = torch.zeros((10,) + cell.shape, dtype=torch.float32, device="cuda")
        cnt = B.of_precond_collect(h, rho, 4, 10, s)
        assert cnt == 10
        s0 = s[0].double().cpu().numpy()
        # the first sample is the right-hand side 4 pi (rho - mean) scaled to unit RMS
        ref = rho.cpu().numpy() - rho.mean().item()
        ref = ref / np.sqrt(np.mean(ref ** 2))
        assert np.abs(s0 - ref).max() <= 1e-6 * np.abs(ref).max()
        # CG residuals shrink in the A^{-1} norm; their RMS falls well below the first one's
        rms = [float(torch.sqrt(torch.mean(s[k].double() ** 2))) for k in range(cnt)]
        assert rms[-1] < 0.5 * rms[0]
    finally:
        B.of_grid_destroy(h)


@pytest.fixture(scope="module")
def trained():
    # residual sets of the 4-atom 32^3 cell and of the 108-atom 96^3 cell (same spacing)
    net, losses = _train([W.al4_cell(), W.al108_cell()], [4, 8])
    yield net, losses
    B.of_precond_destroy(net)


def test_training_lowers_the_loss(trained):
    net, losses = trained
    # mean loss of fixed samples of each cell: lower after training, and negative (better than
    # the zero correction)
    for before, after in losses:
        assert after < before and after < 0, losses


def _solve(cell, rho, opts):
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        phi = torch.zeros_like(rho)
        info = B.of_poisson_solve(h, rho, phi, opts)
        return phi.cpu().numpy(), info
    finally:
        B.of_grid_destroy(h)


def _opts(precision, net=None, no_mg=1, theta=0.3):
    o = B.of_default_solve_opts()
    o.tol = 1e-10
    o.precision = precision
    o.no_multigrid = no_mg
    o.inner_tol = 1e-4
    if net is not None:
        o.precond = net
        o.precond_theta = theta
    return o


def test_trained_network_cuts_iterations_same_answer(trained):
    net, _ = trained
    cell = W.al108_cell()
    rho = _density(cell, cell.n)
    ref, _ = _solve(cell, rho, _opts(B.OF_F64))
    phi_j, info_j = _solve(cell, rho, _opts(B.OF_F32))            # Jacobi (plain) CG inner
    phi_n, info_n = _solve(cell, rho, _opts(B.OF_F32, net))       # flexible CG with the net
    scale = np.abs(ref).max()
    assert info_j.rel_residual <= 1e-10 and info_n.rel_residual <= 1e-10
    assert np.abs(phi_n - ref).max() <= 1e-9 * scale
    assert np.abs(phi_j - ref).max() <= 1e-9 * scale
    assert info_n.net_steps > 0
    # the network's gain: fewer iterations than Jacobi CG to the same true residual (measured
    # 311 against 723 on a GB300; the bar leaves room for training noise)
    assert info_n.iterations < 0.7 * info_j.iterations, (info_n.iterations, info_j.iterations)


def test_refused_network_falls_back_to_plain_cg(trained):
    # a network whose output is negated is never a descent direction: every step is plain, and
    # the count matches Jacobi CG's up to rounding (the flexible CG forms its directions by
    # A-orthogonalisation, plain CG by the Fletcher-Reeves beta: equal in exact arithmetic)
    net, _ = trained
    p = B.of_precond_get_params(net).copy()
    k3 = 7809 - (16 * 27 + 1)
    p[k3:] *= -1.0
    bad = B.of_precond_create(p)
    try:
        cell = W.al4_displaced_cell()
        rho = _density(cell, cell.n)
        _, info_j = _solve(cell, rho, _opts(B.OF_F32))
        phi_b, info_b = _solve(cell, rho, _opts(B.OF_F32, bad))
        assert info_b.net_steps == 0
        assert abs(info_b.iterations - info_j.iterations) <= 2, (info_b.iterations, info_j.iterations)
        assert info_b.rel_residual <= 1e-10
    finally:
        B.of_precond_destroy(bad)


def test_invalid_arguments():
    with pytest.raises(B.OfError):
        B.of_precond_create(np.zeros(10, dtype=np.float32))
    net = B.of_precond_create(_flat(_params(1)))
    h, _ = _grid((16, 16, 16))
    try:
        s = torch.zeros((2, 16, 16, 16), dtype=torch.float32, device="cuda")
        with pytest.raises(B.OfError):
            B.of_precond_train(h, net, s, 2, [0, 5], 1, 2, 1e-3)   # index outside [0, 2)
    finally:
        B.of_grid_destroy(h)
        B.of_precond_destroy(net)
