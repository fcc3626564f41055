"""GPU ground states and forces (C ABI) against the FP64 CPU oracle.

Bars: |E_gpu - E_oracle| <= 1e-6 Ha/atom, forces within 1e-5 Ha/bohr, for the plain FP64
path and the mixed-precision path (FP32 Krylov sweeps with FP64 refinement).  The 32^3
references are stored in tests/golden/ground_states.json, written by
tests/golden/make_golden.py from the oracle alone; the 16^3 cases are computed live.
At the 108-atom, 96^3 size the checks are properties that hold at any size.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
E_TOL = 1e-6   # Ha/atom
F_TOL = 1e-5   # Ha/bohr


def _golden():
    with open(os.path.join(HERE, "golden", "ground_states.json")) as f:
        return json.load(f)


def _run(cell, fn, prec, **kw):
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        o = B.of_default_scf_opts()
        o.precision = prec
        for k, v in kw.items():
            setattr(o, k, v)
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        res = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
        F = B.of_forces(h, sysd, u, phi)
        return res, F, u.cpu().numpy(), phi.cpu().numpy()
    finally:
        B.of_grid_destroy(h)


def _cell_from(rec):
    return W.Cell(n=tuple(rec["n"]), L=tuple(rec["L"]), R=np.array(rec["R"]), Z=np.array(rec["Z"]),
                  sigma=rec["sigma"], rc=rec["rc"], name=rec["name"])


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_tfw_small_cell_live_oracle(prec):
    cell = W.al4_displaced_cell(points_per_cell=16)
    grid = O.Grid(cell.n, cell.L, 6)
    ref = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.tfw_functional(),
                             nlcg_tol=1e-7)
    Fref = O.forces(ref.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    res, F, u, phi = _run(cell, Fn.tfw(), prec)
    assert res.converged
    assert abs(res.energy - ref.energy) / cell.n_atoms <= E_TOL
    for k in ("tf", "vw", "xc", "es", "self", "corr"):
        assert abs(getattr(res, "e_" + k) - ref.terms[k]) / cell.n_atoms <= 1e-5, k
    assert np.max(np.abs(F - Fref)) <= F_TOL
    assert np.max(np.abs(u - ref.u)) <= 1e-4 * ref.u.max()


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_tfw_config1_against_golden(prec):
    rec = _golden()["al4_tfw"]
    cell = _cell_from(rec)
    res, F, u, phi = _run(cell, Fn.tfw(), prec)
    assert res.converged
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL
    # perfect FCC with ions on grid points: forces vanish by symmetry
    assert np.max(np.abs(F)) <= 1e-8
    assert abs(np.sum(u * u) * np.prod(np.array(cell.L) / np.array(cell.n)) - cell.n_electrons) < 1e-10


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_preconditioned_nlcg_reaches_the_golden_minimum(prec):
    # the NLCG preconditioned by one V-cycle of -L_h + 8 on the gradient (Sec. 5.5's real-space
    # preconditioner) ends at the oracle's plain-NLCG minimum, in fewer steps than the plain
    # NLCG on the GPU
    rec = _golden()["al4_tfw"]
    cell = _cell_from(rec)
    plain, _, _, _ = _run(cell, Fn.tfw(), prec)
    res, F, u, phi = _run(cell, Fn.tfw(), prec, nlcg_precond_shift=8.0)
    assert res.converged
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL
    assert res.nlcg_iterations < 0.7 * plain.nlcg_iterations, (res.nlcg_iterations, plain.nlcg_iterations)
    wrec = _golden()["al4_wt"]
    wcell = _cell_from(wrec)
    wres, wF, _, _ = _run(wcell, Fn.wt(), prec, anderson_m=3, anderson_zeta=1.0, nlcg_precond_shift=8.0)
    assert wres.converged
    assert abs(wres.energy - wrec["energy"]) / wcell.n_atoms <= E_TOL
    assert np.max(np.abs(wF - np.array(wrec["forces"]))) <= F_TOL
    # the two-shift form (-L_h + 0.01)(-L_h + 1.5)^{-2}: the same minimum
    for c, r, fn, kw in ((cell, rec, Fn.tfw(), {}), (wcell, wrec, Fn.wt(), dict(anderson_m=3, anderson_zeta=1.0))):
        tres, tF, _, _ = _run(c, fn, prec, nlcg_precond_shift=1.5, nlcg_precond_low=0.01, **kw)
        assert tres.converged
        assert abs(tres.energy - r["energy"]) / c.n_atoms <= E_TOL
        assert np.max(np.abs(tF - np.array(r["forces"]))) <= F_TOL


@pytest.mark.parametrize("prec,inexact", [(B.OF_F64, 0.0), (B.OF_F32, 0.0), (B.OF_F32, 1e-3)])
def test_wt_small_cell_against_golden(prec, inexact):
    rec = _golden()["al4_wt"]
    cell = _cell_from(rec)
    res, F, u, phi = _run(cell, Fn.wt(), prec, nlcg_tol_rel=inexact, anderson_m=3,
                          anderson_zeta=1.0)
    assert res.converged, (res.fp_error, res.nlcg_residual)
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    assert abs(res.e_lr - rec["terms"]["lr"]) / cell.n_atoms <= 1e-5
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_wgc_second_order_kernel_small_cell_live_oracle(prec):
    # full WGC (L = 2, every class of App. A) on the soft-ion 4-atom cell at 16^3
    cell = W.al4_lr_cell(points_per_cell=16)
    grid = O.Grid(cell.n, cell.L, 6)
    ref = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.wgc_functional(),
                             nlcg_tol=1e-8, fp_tol=1e-7, anderson_m=3, zeta=1.0)
    Fref = O.forces(ref.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    res, F, u, phi = _run(cell, Fn.wgc(), prec, nlcg_tol=1e-8, anderson_m=3, anderson_zeta=1.0)
    assert res.converged, (res.fp_error, res.nlcg_residual)
    assert abs(res.energy - ref.energy) / cell.n_atoms <= E_TOL
    assert abs(res.e_lr - ref.terms["lr"]) / cell.n_atoms <= 1e-5
    assert np.max(np.abs(F - Fref)) <= F_TOL


@pytest.mark.parametrize("prec", [B.OF_F64, B.OF_F32])
def test_relaxation_matches_oracle(prec):
    # geometry relaxation (Sec. 3.3): one atom of the 4-atom TFW cell moved by 0.25 bohr, both
    # sides relaxed to max |F| < 1e-5 with the same NLCG / secant steps
    from oracle.relax import relax
    cell = W.al4_cell(points_per_cell=12)
    R0 = cell.R.copy()
    R0[0, 0] += 0.25
    grid = O.Grid(cell.n, cell.L, 6)
    ref = relax(grid, R0, cell.Z, cell.sigma, cell.rc, O.tfw_functional(), ftol=1e-5, nlcg_tol=1e-9)
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        so = B.of_default_scf_opts()
        so.precision = prec
        so.nlcg_tol = 1e-9
        ro = B.of_default_relax_opts()
        ro.ftol = 1e-5
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        R, F, res = B.of_relax(h, B.make_system(R0, cell.Z, cell.sigma, cell.rc), Fn.tfw(), so, ro,
                               u, phi)
    finally:
        B.of_grid_destroy(h)
    assert res.converged and res.max_force < 1e-5 and np.abs(F).max() == res.max_force
    assert res.steps == ref.steps and res.evaluations == ref.evaluations
    assert abs(res.energy - ref.energy) / cell.n_atoms <= E_TOL
    assert np.abs((R - R[0]) - (ref.R - ref.R[0])).max() < 2e-4
    assert np.abs(R - ref.R).max() < 1e-3


@pytest.mark.parametrize("relaxed", [False, True])
def test_vacancy_formation_matches_oracle(relaxed):
    # Sec. 5.6: E_vf = E(M-1, 1, (M-1)/M Omega) - ((M-1)/M) E(M, 0, Omega) for the 8-atom TFW cell
    # (2x1x1 FCC, 12 points per cell edge) with site 0 removed, unrelaxed and relaxed at fixed
    # volume, against the oracle's workflow
    from oracle.vacancy import vacancy_formation
    cell = W.fcc_supercell((2, 1, 1), points_per_cell=12)
    grid = O.Grid(cell.n, cell.L, 6)
    ref = vacancy_formation(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.tfw_functional(), 0,
                            relaxed=relaxed, relax_kw=dict(ftol=1e-4), nlcg_tol=1e-9)
    stream = torch.cuda.current_stream()
    hp = B.of_grid_create(cell.n, cell.L, 6, stream)
    hv = B.of_grid_create(cell.n, B.vacancy_cell_lengths(cell.L, cell.n_atoms), 6, stream)
    try:
        so = B.of_default_scf_opts()
        so.precision = B.OF_F32
        so.nlcg_tol = 1e-9
        ro = None
        if relaxed:
            ro = B.of_default_relax_opts()
            ro.ftol = 1e-4
        up = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        uv = torch.ones_like(up)
        pp, pv = torch.zeros_like(up), torch.zeros_like(up)
        R, res = B.of_vacancy_formation(hp, hv, B.make_system(cell.R, cell.Z, cell.sigma, cell.rc),
                                        0, Fn.tfw(), so, ro, up, pp, uv, pv)
    finally:
        B.of_grid_destroy(hp)
        B.of_grid_destroy(hv)
    M = cell.n_atoms
    assert abs(res.e_perfect - ref.e_perfect) / M <= E_TOL
    assert abs(res.e_unrelaxed - ref.e_unrelaxed) / (M - 1) <= E_TOL
    assert abs(res.evf_unrelaxed - ref.evf_unrelaxed) <= 2 * M * E_TOL
    assert abs(res.evf_relaxed - ref.evf_relaxed) <= 2 * M * E_TOL
    if relaxed:
        assert res.relax_steps == ref.relax_steps and res.evaluations == ref.evaluations
        assert res.max_force < 1e-4 and res.evf_relaxed < res.evf_unrelaxed
        assert np.abs(R - ref.R_vacancy).max() < 1e-3
    else:
        assert res.evf_relaxed == res.evf_unrelaxed and res.relax_steps == 0
        assert np.abs(R - O.vacancy_cell(grid, cell.R, cell.Z, 0)[1]).max() <= 1e-13


def test_vacancy_formation_rejects_a_cell_of_the_wrong_size():
    cell = W.al4_cell(points_per_cell=12)
    stream = torch.cuda.current_stream()
    hp = B.of_grid_create(cell.n, cell.L, 6, stream)
    hv = B.of_grid_create(cell.n, cell.L, 6, stream)   # not scaled to the volume per atom
    try:
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        with pytest.raises(B.OfError) as e:
            B.of_vacancy_formation(hp, hv, sysd, 0, Fn.tfw(), None, None, u, u.clone(), u.clone(),
                                   u.clone())
        assert e.value.status == B.OF_EINVAL
        with pytest.raises(B.OfError):
            B.of_vacancy_formation(hp, hv, sysd, 4, Fn.tfw(), None, None, u, u.clone(), u.clone(),
                                   u.clone())
    finally:
        B.of_grid_destroy(hp)
        B.of_grid_destroy(hv)


def test_fixed_point_on_u_matches_golden():
    # the alternative fixed point of Sec. 5.3 (Anderson mixing of u instead of V_LR) reaches
    # the same ground state
    rec = _golden()["al4_wt"]
    cell = _cell_from(rec)
    res, F, u, phi = _run(cell, Fn.wt(), B.OF_F32, anderson_m=3, anderson_zeta=1.0,
                          fixed_point=B.OF_FP_U)
    assert res.converged, (res.fp_error, res.nlcg_residual)
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL


def test_vw_energy_gradient_form():
    # the vW energy reported as (lam/2) int |grad_h u|^2 (Eq. gradient:approximate) instead of
    # -(lam/2) <u, L_h u>: same ground state, the term is the gradient form's integral of the
    # returned u (order-12 first-difference weights from the oracle), and the two forms differ
    # only by the discretisation error
    rec = _golden()["al4_tfw"]
    cell = _cell_from(rec)
    res_l, _, u_l, _ = _run(cell, Fn.tfw(), B.OF_F64)
    res_g, _, u_g, phi_g = _run(cell, Fn.tfw(), B.OF_F64, vw_energy=B.OF_VW_GRADIENT)
    grid = O.Grid(cell.n, cell.L, 6)
    grad_sq = np.zeros_like(u_g)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        w = O.fd_gradient_weights(6, grid.h[a])
        g = sum(w[p] * (np.roll(u_g, -p, axis=ax) - np.roll(u_g, p, axis=ax)) for p in range(1, 7))
        grad_sq += g * g
    vw = 0.5 * O.tfw_functional().lam * np.sum(grad_sq) * grid.dV
    assert abs(res_g.e_vw - vw) <= 1e-11 * abs(vw)
    assert abs(res_g.e_tf - res_l.e_tf) <= 1e-9 * abs(res_l.e_tf)
    assert abs(res_g.e_vw - res_l.e_vw) <= 1e-3 * abs(res_l.e_vw)


def test_line_searches_reach_the_same_ground_state():
    # Brent on the energy (the paper's line search) and the slope search (root of dE/ds from
    # the same line model) stop the NLCG at the same minimiser; the slope search needs fewer
    # passes per NLCG step.  A wrong term in dE/ds would move its root off the energy minimum
    # and fail the golden bars or stall the NLCG.
    rec = _golden()["al4_wt"]
    cell = _cell_from(rec)
    out = {}
    for line in (B.OF_LINE_BRENT, B.OF_LINE_SLOPE):
        res, F, u, phi = _run(cell, Fn.wt(), B.OF_F32, line_search=line, anderson_m=3,
                              anderson_zeta=1.0)
        assert res.converged, (line, res.fp_error, res.nlcg_residual)
        assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
        assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL
        out[line] = res
    rb, rs = out[B.OF_LINE_BRENT], out[B.OF_LINE_SLOPE]
    assert abs(rb.energy - rs.energy) / cell.n_atoms <= 1e-8
    per_step = {k: r.line_evaluations / max(1, r.nlcg_iterations) for k, r in out.items()}
    assert per_step[B.OF_LINE_SLOPE] < 0.6 * per_step[B.OF_LINE_BRENT], per_step


def _bench_like_opts(o):
    # the benchmark's options (bench.make_case): Anderson m = 3, zeta = 1, fixed point to 1e-6,
    # inexact inner solves (NLCG to 0.03 x the previous fixed-point error, FP32 Poisson passes
    # to 3e-4)
    o.fp_tol = 1e-6
    o.anderson_m = 3
    o.anderson_zeta = 1.0
    o.nlcg_tol_rel = 3e-2
    o.poisson.inner_tol = 3e-4
    o.nlcg_precond_shift = 1.5   # the chosen form's NLCG preconditioner,
    o.nlcg_precond_low = 0.01    # (-L_h + 0.01)(-L_h + 1.5)^{-2}
    return o


def test_wt_small_cell_with_the_benchmark_options_against_golden():
    rec = _golden()["al4_wt"]
    cell = _cell_from(rec)
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    try:
        sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
        o = _bench_like_opts(B.of_default_scf_opts())
        o.precision = B.OF_F32
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        res = B.of_scf_ground_state(h, sysd, Fn.wt(), o, u, phi)
        F = B.of_forces(h, sysd, u, phi)
    finally:
        B.of_grid_destroy(h)
    assert res.converged
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL


@pytest.mark.parametrize("form", ["mixed", "f64"])
def test_benchmark_cell_against_the_oracle(form):
    # the benchmark step itself -- 108 atoms, 96^3, WT-type kernel, exactly bench.make_case's
    # options and call sequence -- against the oracle's ground state of the same cell
    # (tests/golden/al108_wt.json, written by tests/golden/make_golden.py from the oracle alone)
    import bench
    path = os.path.join(HERE, "golden", "al108_wt.json")
    with open(path) as f:
        rec = json.load(f)["al108_wt"]
    cell, h, sysd, fn, o = bench.make_case(torch, B, Fn, W, form)
    try:
        assert np.array_equal(np.array(rec["R"]), cell.R)       # same seeded positions
        assert rec["sigma"] == cell.sigma and rec["rc"] == cell.rc and list(rec["n"]) == list(cell.n)
        u0 = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        u = torch.empty_like(u0)
        phi = torch.zeros_like(u0)
        res, F = bench.run_step(B, h, sysd, fn, o, u, phi, u0)
    finally:
        B.of_grid_destroy(h)
    assert res.converged
    assert abs(res.energy - rec["energy"]) / cell.n_atoms <= E_TOL
    for k in ("tf", "vw", "lr", "xc", "es", "self", "corr"):
        assert abs(getattr(res, "e_" + k) - rec["terms"][k]) / cell.n_atoms <= 1e-5, k
    assert np.max(np.abs(F - np.array(rec["forces"]))) <= F_TOL


def test_wt_108_atoms_full_size_properties():
    cell = W.al108_cell()
    res, F, u, phi = _run(cell, Fn.wt(), B.OF_F32, fp_tol=1e-6)
    assert res.converged
    dV = np.prod(np.array(cell.L) / np.array(cell.n))
    assert abs(np.sum(u * u) * dV - cell.n_electrons) < 1e-9 * cell.n_electrons
    assert u.min() > 0
    assert abs(phi.mean()) < 1e-10 * np.abs(phi).max()
    # momentum balance of the Hellmann-Feynman forces (broken only by the grid)
    assert np.max(np.abs(F.sum(0))) < 1e-4
    # the ground state lies below the uniform-density energy reached before any update
    assert res.energy < 0


def test_batched_ground_states_match_single_cell_calls():
    # three different cells in one call (stream pool): each equals its own single-cell ground
    # state, and the first equals the oracle's
    cells = [W.al4_displaced_cell(points_per_cell=16), W.al4_cell(points_per_cell=16),
             W.small_cell(n=(16, 20, 18), L=(7.6, 9.5, 8.55), seed=3)]
    stream = torch.cuda.current_stream()
    grids = [B.of_grid_create(c.n, c.L, 6, stream) for c in cells]
    try:
        systems = [B.make_system(c.R, c.Z, c.sigma, c.rc) for c in cells]
        o = B.of_default_scf_opts()
        o.precision = B.OF_F32
        us = [torch.ones(c.shape, dtype=torch.float64, device="cuda") for c in cells]
        phis = [torch.zeros_like(x) for x in us]
        results = B.of_scf_ground_state_batched(grids, systems, Fn.tfw(), o, us, phis)
        for k, c in enumerate(cells):
            assert results[k].converged, k
            u1 = torch.ones(c.shape, dtype=torch.float64, device="cuda")
            p1 = torch.zeros_like(u1)
            one = B.of_scf_ground_state(grids[k], systems[k], Fn.tfw(), o, u1, p1)
            assert abs(results[k].energy - one.energy) / c.n_atoms <= 1e-8, k
            assert torch.max(torch.abs(us[k] - u1)).item() <= 1e-5 * torch.max(u1).item(), k
        grid = O.Grid(cells[0].n, cells[0].L, 6)
        ref = O.scf_ground_state(grid, cells[0].R, cells[0].Z, cells[0].sigma, cells[0].rc,
                                 O.tfw_functional(), nlcg_tol=1e-7)
        assert abs(results[0].energy - ref.energy) / cells[0].n_atoms <= E_TOL
    finally:
        for g in grids:
            B.of_grid_destroy(g)


def test_ground_states_are_bitwise_reproducible():
    # every reduction sums in a fixed order and the nuclear charge is gathered, not scattered:
    # the same WT ground state with the benchmark's options (twin handles, concurrent kernel-map
    # solves, the two-shift NLCG preconditioner) on two handles, and inside a batched call
    # beside another cell, gives the same bits
    cell = W.al4_lr_cell(points_per_cell=16)
    other = W.fcc_supercell((1, 1, 1), points_per_cell=16, displacement=0.05, seed=7, sigma=1.2, rc=10.0)
    stream = torch.cuda.current_stream()
    o = _bench_like_opts(B.of_default_scf_opts())
    o.precision = B.OF_F32
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    runs = []
    for _ in range(2):
        h = B.of_grid_create(cell.n, cell.L, 6, stream)
        try:
            u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
            phi = torch.zeros_like(u)
            res = B.of_scf_ground_state(h, sysd, Fn.wt(), o, u, phi)
            runs.append((res.energy, u, B.of_forces(h, sysd, u, phi)))
        finally:
            B.of_grid_destroy(h)
    grids = [B.of_grid_create(c.n, c.L, 6, stream) for c in (other, cell)]
    try:
        us = [torch.ones(c.shape, dtype=torch.float64, device="cuda") for c in (other, cell)]
        phis = [torch.zeros_like(x) for x in us]
        systems = [B.make_system(other.R, other.Z, other.sigma, other.rc), sysd]
        results = B.of_scf_ground_state_batched(grids, systems, Fn.wt(), o, us, phis)
    finally:
        for g in grids:
            B.of_grid_destroy(g)
    assert runs[0][0] == runs[1][0] == results[1].energy
    assert torch.equal(runs[0][1], runs[1][1]) and torch.equal(runs[0][1], us[1])
    assert np.array_equal(runs[0][2], runs[1][2])


def test_batched_wt_ground_states_of_uneven_cells_match_the_oracle():
    # the batched call on cells of different shapes and atom counts, one with a vacancy, with
    # the WT-type kernel term and the benchmark's options: every cell's energy and forces
    # against the oracle's own ground state of that cell
    cells = [W.fcc_supercell((1, 1, 1), points_per_cell=16, displacement=0.1, seed=11,
                             sigma=1.2, rc=10.0, name="c111"),
             W.fcc_supercell((2, 1, 1), points_per_cell=12, displacement=0.1, seed=12,
                             vacancy="random", sigma=1.2, rc=10.0, name="c211v"),
             W.fcc_supercell((1, 2, 1), points_per_cell=12, displacement=0.1, seed=13,
                             sigma=1.2, rc=10.0, name="c121")]
    stream = torch.cuda.current_stream()
    grids = [B.of_grid_create(c.n, c.L, 6, stream) for c in cells]
    try:
        systems = [B.make_system(c.R, c.Z, c.sigma, c.rc) for c in cells]
        o = _bench_like_opts(B.of_default_scf_opts())
        o.precision = B.OF_F32
        us = [torch.ones(c.shape, dtype=torch.float64, device="cuda") for c in cells]
        phis = [torch.zeros_like(x) for x in us]
        results = B.of_scf_ground_state_batched(grids, systems, Fn.wt(), o, us, phis)
        for k, c in enumerate(cells):
            assert results[k].converged, c.name
            F = B.of_forces(grids[k], systems[k], us[k], phis[k])
            grid = O.Grid(c.n, c.L, 6)
            ref = O.scf_ground_state(grid, c.R, c.Z, c.sigma, c.rc, O.wt_functional(),
                                     nlcg_tol=1e-7, fp_tol=1e-7, anderson_m=3, zeta=1.0)
            Fref = O.forces(ref.phi, c.R, c.Z, c.sigma, c.rc, grid)
            assert abs(results[k].energy - ref.energy) / c.n_atoms <= E_TOL, c.name
            assert np.max(np.abs(F - Fref)) <= F_TOL, c.name
    finally:
        for g in grids:
            B.of_grid_destroy(g)
