#!/usr/bin/env python3
"""Benchmark of the periodic OF-DFT hot path on one GB300 (or N independent replicas).

Step = one complete ground state of the 108-atom 3x3x3 FCC Al-like cell (a = 7.6 bohr,
+-0.1 bohr seeded displacements, Gaussian ions Z = 3), 96^3 grid, 12th-order FD, WT-type
kernel functional, followed by the forces: of_scf_ground_state + of_forces through the C
ABI.  The chosen form runs the Poisson and kernel solves as FP32 Krylov sweeps with FP64
iterative refinement (Poisson inner CG preconditioned by a multigrid V-cycle); --precision
f64 runs the plain FP64 CG form.  The working set (~0.4 GB) sits in L2 between kernels of one
step, so L2 is flushed (a 256 MiB write) between timed steps, outside the timed events.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded sample of
the same workload instead (see cpu_baseline).
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per SCF ground state & stencil GPts/s: chosen vs plain FP64 CG, at 1e-6 Ha/atom"
UNIT = "s/ground-state"
NLCG_PRECOND_SHIFT = 1.5   # bohr^-2
NLCG_PRECOND_LOW = 0.01    # bohr^-2
POISSON_PASS_TOL = 3e-4    # each FP32 Poisson pass stops at this fraction of its start residual
WORKLOAD = ("108-atom FCC Al-like cell (3x3x3, a=7.6 bohr, +-0.1 bohr displacements, seed 2), "
            "96^3 grid, 12th-order FD, WT-type kernel functional, ground state + forces")
# what else defines the step (the options of make_case)
WORKLOAD_DETAIL = {
    "ions": "normalised Gaussian pseudocharges Z=3, sigma=1.2 bohr, r_c=10 bohr (sigma=0.7 "
            "gives the kernel functional no minimiser with u >= 0)",
    "functional": "TF + vW (lambda=1) + WT-type kernel (mu=1, alpha,beta=(5+-sqrt5)/6, the "
                  "K_00 rows of the WGC table) + PZ LDA",
    "anderson": {"m": 3, "zeta": 1.0, "fixed_point_tol": 1e-6, "variable": "V_LR"},
    "nlcg": {"tol": 1e-7, "line_search": "root of dE/ds (secant), line_tol 1e-3",
             "inexact": "NLCG of outer step k stops at max(1e-7, 0.03 x fixed-point error of "
                        "step k-1); the last outer step at 1e-7",
             "preconditioner": "chosen form: (-L_h + 0.01) (-L_h + 1.5)^-2 on the gradient (two "
                               "multigrid V-cycles and one FP32 sweep), preconditioned "
                               "Polak-Ribiere (the real-space NLCG preconditioner Sec. 5.5 calls "
                               "for); plain FP64 form: none"},
    "poisson": {"tol": 1e-10, "form": "FP32 multigrid-preconditioned CG passes to 3e-4 of "
                                      "their starting residual, FP64 refinement"},
    "kernel_solves": {"form": "FP32 COCG preconditioned by the V-cycle of -L + kf2 |Q|, FP64 "
                              "refinement", "tol": "max(1e-10, min(1e-5, 1e-2 x previous "
                                                  "fixed-point error))"},
}
GOLDEN_AL108 = os.path.join(ROOT, "tests", "golden", "al108_wt.json")
# DRAM bytes (read + write) of one FP32 order-12 sweep of a 320^3 grid by the fast-path stencil,
# from the ncu capture summarised in profiles/stencil_fp32_320.md (145.9 + 91.9 MB)
STENCIL320_DRAM_BYTES = 237.8e6
# DRAM bytes that one V-cycle plus one COCG iteration of the 96^3 complex FP32 pass moves,
# summed over its kernels launched one by one from a cold L2 (ncu; the kernels' table is in
# profiles/mg_cocg_pass_kernels_96.md)
COCG96_DRAM_BYTES_PER_ITERATION = 167e6
# algorithmic FP64 arithmetic of one order-12 Laplacian point: 3 axes x 12 neighbours + the
# centre, one multiply-add (2 flops) each
STENCIL_F64_FLOPS_PER_POINT = 2 * (3 * 12 + 1)
GOLDEN_SMALL = os.path.join(ROOT, "tests", "golden", "ground_states.json")


def golden_al108():
    """The oracle's ground state of this workload (tests/golden/al108_wt.json, written by
    tests/golden/make_golden.py from the oracle alone), or None if absent."""
    if not os.path.exists(GOLDEN_AL108):
        return None
    with open(GOLDEN_AL108) as f:
        return json.load(f)["al108_wt"]


def oracle_counts():
    """NLCG steps and kernel maps (one per outer iteration) of the oracle's own ground state of
    this workload, from its stored record: the constants that scale the oracle's timed sample
    to one ground state."""
    rec = golden_al108()
    if rec is None:
        raise RuntimeError("tests/golden/al108_wt.json is missing: run "
                           "python tests/golden/make_golden.py --al108")
    return int(sum(rec["nlcg_iterations"])), int(rec["outer_iterations"])


def errors_vs_oracle(res, F, n_atoms):
    """Energy (Ha/atom) and largest force-component (Ha/bohr) difference from the oracle's
    stored ground state of this workload."""
    import numpy as np
    rec = golden_al108()
    if rec is None:
        return None
    return {"energy_error_vs_oracle_ha_per_atom": abs(res.energy - rec["energy"]) / n_atoms,
            "max_force_error_vs_oracle_ha_per_bohr": float(np.max(np.abs(F - np.array(rec["forces"])))),
            "oracle_energy_per_atom_ha": rec["energy_per_atom"],
            "tolerances": {"energy_ha_per_atom": 1e-6, "force_ha_per_bohr": 1e-5}}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    p.add_argument("--no-compare-f64", action="store_true",
                   help="skip the plain FP64 CG ground state (same options) timed beside the step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--config3", action="store_true",
                   help="batched ground states of the first --cells cells of the 64-cell set")
    p.add_argument("--cells", type=int, default=64)
    p.add_argument("--config5", action="store_true",
                   help="measure the 3999-atom 320^3 ground state instead of the benchmark step")
    p.add_argument("--wgc", action="store_true",
                   help="measure the 108-atom 96^3 ground state with the full WGC functional "
                        "(second-order kernel expansion) instead of the benchmark step")
    p.add_argument("--relax", action="store_true",
                   help="measure a geometry relaxation of the 108-atom 96^3 cell instead of the "
                        "benchmark step")
    p.add_argument("--convergence", action="store_true",
                   help="mesh convergence of the energy and forces with the FD order (4-atom "
                        "cell, orders 2, 6, 12) instead of the benchmark step")
    p.add_argument("--vacancy", action="store_true",
                   help="vacancy formation energy of the 108-atom 96^3 cell (unrelaxed and "
                        "relaxed) instead of the benchmark step")
    p.add_argument("--mixing-study", action="store_true",
                   help="fixed point on V_LR vs on u, Anderson m and zeta, on the 108-atom cell")
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-preconditioner comparison (864-atom 192^3 Poisson)")
    p.add_argument("--no-other-configs", action="store_true",
                   help="skip the other workloads of the default line (3999-atom cell, full WGC, "
                        "relaxation, vacancy formation)")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the 64-cell batched-vs-sequential comparisons (Poisson solves and "
                        "ground states)")
    p.add_argument("--kernel-case", default=None, choices=["poisson96", "stencil96", "stencil320", "scf", "net160", "scf96_short"],
                   help="run only a bounded piece of the step (for profiler captures) and exit: "
                        "poisson96 = 4 mixed Poisson solves on the benchmark grid; stencil96 / "
                        "stencil320 = FP32/FP64 Laplacian sweeps on a 96^3 / 320^3 grid; scf = one "
                        "ground state")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples: $OF_CLOCKS_DIR if set (to keep them), else the temporary directory
        out_dir = os.environ.get("OF_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"of_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_case(torch, B, Fn, W, precision):
    cell = W.al108_cell()
    stream = torch.cuda.current_stream()
    h = B.of_grid_create(cell.n, cell.L, 6, stream)
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    fn = Fn.wt()
    o = B.of_default_scf_opts()
    o.precision = B.OF_F32 if precision == "mixed" else B.OF_F64
    o.fp_tol = 1e-6
    o.anderson_m = 3       # the paper's choice for linear-response runs (Sec. 5.3)
    o.anderson_zeta = 1.0
    # inexact inner solves while the fixed point is far from converged: each outer step's NLCG
    # stops at 0.03 x the previous fixed-point error (the last one at the full tolerance), and
    # each FP32 Poisson pass at 3e-4 of its starting residual (tuned on this cell; with the
    # preconditioned NLCG below, NLCG factors 0.3 / 0.1 / 0.03 / 0.01 gave 0.62 / 0.37 / 0.36 /
    # 0.41 s per ground state, the same energy to 1e-11 Ha/atom; 0.05 / 0.03 / 0.015 later gave
    # 0.303 / 0.281 / 0.331 s; Poisson pass floors 1e-4 / 3e-4 / 1e-3 / 3e-3 gave 0.2817 /
    # 0.2797 / 0.2810 / 0.2859 s, and line_tol 1e-3 / 3e-3 / 1e-2 / 3e-2 0.281 / 0.281 / 0.304 /
    # 0.284 s)
    o.nlcg_tol_rel = 3e-2
    o.poisson.inner_tol = POISSON_PASS_TOL
    # the chosen form preconditions the NLCG with (-L_h + 0.01)(-L_h + 1.5)^{-2} on the
    # gradient, two V-cycles and one sweep, which follows the energy's curvature both at large
    # wave numbers (~k^2, vW) and at small ones (~16 pi rho_bar / k^2, Hartree).  Tuned on this
    # cell and on the 3999-atom cell (s per ground state, 108 / 3999 atoms): one V-cycle of
    # -L_h + 8: 0.328 / 18.3; two-shift (1.5, 0.01): 0.325 / 12.4; (1.5, 0.02): 0.323 / 14.6;
    # (1.2, 0.02): 0.327 / 15.5; (2.0, 0.05): 0.371 / 14.3; without: 0.79 / 27.0.  The plain FP64
    # form keeps the paper's unpreconditioned NLCG
    o.nlcg_precond_shift = NLCG_PRECOND_SHIFT if precision == "mixed" else 0.0
    o.nlcg_precond_low = NLCG_PRECOND_LOW if precision == "mixed" else 0.0
    return cell, h, sysd, fn, o


def run_step(B, h, sysd, fn, o, u, phi, u0):
    u.copy_(u0)
    res = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
    F = B.of_forces(h, sysd, u, phi)
    return res, F


def alu_peaks(B, torch):
    """Measured FMA rates of the CUDA cores (TFLOP/s): FP64, FP32 and packed FP32x2."""
    s = torch.cuda.current_stream()
    return {"fp64_tflops": B.of_alu_peak(B.OF_PEAK_F64, s) / 1e12,
            "fp32_tflops": B.of_alu_peak(B.OF_PEAK_F32, s) / 1e12,
            "fp32x2_tflops": B.of_alu_peak(B.OF_PEAK_F32X2, s) / 1e12}


def stencil_rates(torch, B, shape, L, reps=30):
    """Device time of one of_laplacian_apply sweep (FP32 and FP64) on this grid: `reps` sweeps
    captured in one CUDA graph on a grid handle of their own, replayed between CUDA events
    (host launch overhead excluded).  At 96^3 consecutive sweeps keep the fields in L2; at
    320^3 each FP32 field (131 MB) is larger than L2, so the sweeps stream from HBM.  GB/s
    counts the algorithmic traffic (read x, write y); frac is that over the measured HBM peak."""
    out = {}
    s = torch.cuda.Stream()
    h = B.of_grid_create(shape, L, 6, s)
    try:
        for dt, tdt, name in [(B.OF_F32, torch.float32, "f32"), (B.OF_F64, torch.float64, "f64")]:
            x = torch.rand(shape, dtype=tdt, device="cuda")
            y = torch.empty_like(x)
            torch.cuda.synchronize()
            for _ in range(5):
                B.of_laplacian_apply(h, dt, x, y)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
                for _ in range(reps):
                    B.of_laplacian_apply(h, dt, x, y)
            graph.replay()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            n = x.numel()
            gbs = 2 * n * x.element_size() / (ms * 1e-3) / 1e9
            out[name] = {"gpts": n / (ms * 1e-3) / 1e9, "ms": ms, "gbs": gbs,
                         "frac_of_hbm": gbs / measured_peaks()[0]}
            del graph
    finally:
        torch.cuda.synchronize()
        B.of_grid_destroy(h)
    return out


def batched_compare(torch, B, W, reps=2):
    """64 uneven cells (reps 2..4 per axis, 64-128 points per axis, half with a vacancy, seed 3):
    the Poisson problem of each cell's initial density (uniform electrons plus its Gaussian
    nuclear charge), solved to relative residual 1e-10 by (a) one batched call of grouped
    launches (plain FP32 CG + FP64 refinement), (b) one batched call in the multigrid form
    (per-cell multigrid PCG over concurrent streams), (c) the single-grid solver cell by cell
    with the same plain CG, (d) cell by cell with the multigrid-preconditioned CG."""
    cells = W.batched_cells()
    stream = torch.cuda.current_stream()
    grids, rhos, phis = [], [], []
    for c in cells:
        g = B.of_grid_create(c.n, c.L, 6, stream)
        b = torch.empty(c.shape, dtype=torch.float64, device="cuda")
        B.of_pseudocharge(g, B.make_system(c.R, c.Z, c.sigma, c.rc), b)
        vol = c.L[0] * c.L[1] * c.L[2]
        rhos.append(b + c.n_electrons / vol)
        phis.append(torch.zeros(c.shape, dtype=torch.float64, device="cuda"))
        grids.append(g)
    o = B.of_default_solve_opts()
    o.precision = B.OF_F32
    o.tol = 1e-10
    o.no_multigrid = 1
    om = B.of_default_solve_opts()
    om.precision = B.OF_F32
    om.tol = 1e-10

    def run_batched():
        for p in phis:
            p.zero_()
        return B.of_poisson_solve_batched(grids, rhos, phis, o)

    def run_seq(opts):
        for g, r, p in zip(grids, rhos, phis):
            p.zero_()
            B.of_poisson_solve(g, r, p, opts)

    def run_batched_mg():
        for p in phis:
            p.zero_()
        return B.of_poisson_solve_batched(grids, rhos, phis, om)

    out = {}
    run_batched()   # tunes the blocking, captures the graph
    run_batched_mg()
    run_seq(o)
    run_seq(om)
    for name, fn in [("batched_plain_cg_s", run_batched),
                     ("batched_multigrid_concurrent_s", run_batched_mg),
                     ("sequential_plain_cg_s", lambda: run_seq(o)),
                     ("sequential_multigrid_pcg_s", lambda: run_seq(om))]:
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.time()
            fn()
            torch.cuda.synchronize()
            ts.append(time.time() - t)
        out[name] = min(ts)
    out["cells"] = len(cells)
    out["points"] = int(sum(c.n_points for c in cells))
    out["atoms"] = int(sum(c.n_atoms for c in cells))
    for g in grids:
        B.of_grid_destroy(g)
    return out


def _initial_density(torch, B, cell):
    """Uniform electrons plus the cell's Gaussian nuclear charge: the density of the first
    Poisson solve of a ground-state run."""
    g = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    b = torch.empty(cell.shape, dtype=torch.float64, device="cuda")
    B.of_pseudocharge(g, B.make_system(cell.R, cell.Z, cell.sigma, cell.rc), b)
    B.of_grid_destroy(g)
    return b + cell.n_electrons / (cell.L[0] * cell.L[1] * cell.L[2])


def learned_compare(torch, B, W, steps=400, theta=0.3):
    """Learned preconditioner: trained on the GPU on CG residuals of the Poisson problems of the
    4-atom 32^3 and the 108-atom 96^3 cells (64 residuals each; four Adam runs per cell, batch
    4), then used in the FP32 flexible CG of the Poisson solve of the 864-atom 6x6x6 cell,
    192^3 grid, same spacing, to true relative residual 1e-10; against the same solve with
    plain (Jacobi) FP32 CG, plain FP64 CG and multigrid-preconditioned FP32 CG."""
    import numpy as np
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.time()
    net = B.of_precond_create(W.initial_network(0))
    data = []
    for cell, stride in ((W.al4_cell(), 4), (W.al108_cell(), 8)):
        rho = _initial_density(torch, B, cell)
        g = B.of_grid_create(cell.n, cell.L, 6, stream)
        s = torch.empty((64,) + cell.shape, dtype=torch.float32, device="cuda")
        data.append((g, s, B.of_precond_collect(g, rho, stride, 64, s)))
    rng = np.random.default_rng(0)
    for rnd in range(4):
        for g, s, cnt in data:
            st = steps // 4
            B.of_precond_train(g, net, s, cnt, rng.integers(0, cnt, size=st * 4), st, 4,
                               3e-3 if rnd < 3 else 1e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    for g, _, _ in data:
        B.of_grid_destroy(g)
    del data
    cell = W.al864_cell()
    rho = _initial_density(torch, B, cell)
    g = B.of_grid_create(cell.n, cell.L, 6, stream)
    phi = torch.zeros_like(rho)

    def opts(prec, no_mg, use_net):
        o = B.of_default_solve_opts()
        o.tol, o.precision, o.no_multigrid, o.inner_tol = 1e-10, prec, no_mg, 1e-4
        if use_net:
            o.precond, o.precond_theta = net, theta
        return o

    out = {"workload": "al864 Poisson (uniform density + ions), 192^3, tol 1e-10",
           "training_s": train_s, "training_steps": steps, "theta": theta}
    for name, o in (("jacobi_cg_mixed", opts(B.OF_F32, 1, False)),
                    ("learned_fcg_mixed", opts(B.OF_F32, 1, True)),
                    ("plain_cg_f64", opts(B.OF_F64, 1, False)),
                    ("multigrid_pcg_mixed", opts(B.OF_F32, 0, False))):
        phi.zero_()
        B.of_poisson_solve(g, rho, phi, o)     # workspace, graphs
        phi.zero_()
        torch.cuda.synchronize()
        t = time.time()
        info = B.of_poisson_solve(g, rho, phi, o)
        torch.cuda.synchronize()
        out[name] = {"s": time.time() - t, "iterations": info.iterations,
                     "refinements": info.refinements, "network_steps": info.net_steps,
                     "rel_residual": info.rel_residual}
    out["shifted"] = learned_shifted_compare(torch, B, W, g, cell, steps, theta)
    r = torch.randn(cell.shape, dtype=torch.float32, device="cuda")
    z = torch.empty_like(r)
    B.of_precond_apply(g, net, r, z)
    torch.cuda.synchronize()
    t = time.time()
    for _ in range(10):
        B.of_precond_apply(g, net, r, z)
    torch.cuda.synchronize()
    out["network_apply_ms"] = (time.time() - t) / 10 * 1e3
    B.of_grid_destroy(g)
    B.of_precond_destroy(net)
    return out


def _kernel_rhs(torch, B, W, g, cell, kf2, seed):
    """A kernel-map right-hand side f = -(1/kf2) L_h q (the m = n = 0 form of Sec. 3.1) of a
    smooth positive seeded field q standing in for u^{2 alpha}, formed on the device."""
    q = torch.from_numpy(1.0 + 0.5 * W.random_field(cell.shape, seed=seed, kind="smooth")).cuda()
    f = torch.empty_like(q)
    B.of_laplacian_apply(g, B.OF_F64, q, f)
    return f * (-1.0 / kf2)


def learned_shifted_compare(torch, B, W, g864, cell864, steps, theta):
    """The learned preconditioner for a shifted kernel system: a network trained for the real
    operator -L_h + c, c = kf2 |Q| of the WT kernel's second shift (Q = 0.066 - 0.260i), on
    every CG residual of that real system on the 108-atom 96^3 cell (four right-hand sides,
    2 x steps Adam steps), then used in the inner flexible CG on that operator that preconditions
    the FP32 flexible GMRES(8) of the same shifted system on the 864-atom 192^3 grid (a
    right-hand side not trained on) to true relative residual 1e-10; against the same solver
    with every network step refused (plain inner CG), plain FP32 COCG, plain FP64 COCG and
    multigrid-preconditioned FP32 COCG.  Iterations count the inner steps too."""
    import numpy as np
    from paper_1412_8250_gb300 import functionals as Fn
    fn = Fn.wt()
    Pk, Qk = complex(fn.P[4], fn.P[5]), complex(fn.Q[4], fn.Q[5])
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.time()
    cell = W.al108_cell()
    kf2 = Fn.kf2(cell.n_electrons, float(np.prod(cell.L)))
    c = kf2 * abs(Qk)
    net = B.of_precond_create(W.initial_network(4))
    B.of_precond_set_shift(net, c)
    g = B.of_grid_create(cell.n, cell.L, 6, stream)
    sets = []
    for seed in (41, 43, 45, 49):
        s = torch.empty((48,) + cell.shape, dtype=torch.float32, device="cuda")
        cnt = B.of_precond_collect(g, _kernel_rhs(torch, B, W, g, cell, kf2, seed), 1, 48, s, shift=c)
        sets += [s[k] for k in range(cnt)]
    S = torch.stack(sets).contiguous()
    cnt = S.shape[0]
    rng = np.random.default_rng(4)
    for rnd in range(4):
        st = 2 * steps // 4
        B.of_precond_train(g, net, S, cnt, rng.integers(0, cnt, size=st * 4), st, 4,
                           3e-3 if rnd < 3 else 1e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    B.of_grid_destroy(g)
    del sets
    kf2_864 = Fn.kf2(cell864.n_electrons, float(np.prod(cell864.L)))
    f = _kernel_rhs(torch, B, W, g864, cell864, kf2_864, 47)
    Wc = torch.zeros(cell864.shape + (2,), dtype=torch.float64, device="cuda")

    def opts(prec, no_mg, use_net, th=theta):
        o = B.of_default_solve_opts()
        o.tol, o.precision, o.no_multigrid, o.inner_tol = 1e-10, prec, no_mg, 1e-4
        if use_net:
            o.precond, o.precond_theta = net, th
        return o

    out = {"workload": "al864 shifted kernel system -(1/kf2) L_h W + Q W = P f, Q = 0.066 - 0.260i "
                       "(the WT kernel's second shift), 192^3, tol 1e-10",
           "network_shift_c": c, "training_s": train_s, "training_steps": 2 * steps,
           "training_data": "%d CG residuals of -L_h + c on the 108-atom 96^3 cell, four "
                            "right-hand sides" % cnt}
    for name, o in (("plain_cocg_mixed", opts(B.OF_F32, 1, False)),
                    ("learned_fgmres_mixed", opts(B.OF_F32, 1, True)),
                    ("fgmres_plain_inner_cg_mixed", opts(B.OF_F32, 1, True, 2.0)),
                    ("plain_cocg_f64", opts(B.OF_F64, 1, False)),
                    ("multigrid_pcocg_mixed", opts(B.OF_F32, 0, False))):
        Wc.zero_()
        B.of_kernel_solve(g864, f, [Pk], [Qk], kf2_864, Wc, o)     # workspace, graphs
        Wc.zero_()
        torch.cuda.synchronize()
        t = time.time()
        info = B.of_kernel_solve(g864, f, [Pk], [Qk], kf2_864, Wc, o)
        torch.cuda.synchronize()
        out[name] = {"s": time.time() - t, "iterations": info.iterations,
                     "refinements": info.refinements, "network_steps": info.net_steps,
                     "rel_residual": info.rel_residual}
    B.of_precond_destroy(net)
    return out


def cpu_setup(cell):
    """The oracle's once-per-ground-state work on this cell, timed: nuclear charge, its
    potential, self energy and overlap correction; and the forces (whose cost does not depend
    on the potential's values).  Returns (state, setup seconds, forces seconds)."""
    import numpy as np
    import oracle as O
    t0 = time.time()
    grid = O.Grid(cell.n, cell.L, 6)
    b = O.pseudocharge(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    phib = O.poisson_solve(b, grid)
    O.self_energy(cell.R, cell.Z, cell.sigma, cell.rc, grid)
    O.repulsive_correction(cell.R, cell.Z, cell.sigma, grid.L)
    t_setup = time.time() - t0
    t1 = time.time()
    O.forces(phib, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    t_forces = time.time() - t1
    Ne = cell.n_electrons
    u = np.full(grid.shape, np.sqrt(Ne / grid.volume))
    return (grid, b, phib, u), t_setup, t_forces


def cpu_iteration(cell, state, nlcg_steps=1):
    """One kernel map V[u] and `nlcg_steps` NLCG steps of the oracle on this cell, timed.
    Returns (seconds per kernel map, seconds per NLCG step, state with the advanced u)."""
    import numpy as np
    import oracle as O
    grid, b, phib, u = state
    Ne = cell.n_electrons
    fn = O.wt_functional()
    kf2 = O.kf2_of(Ne, grid.volume)
    t1 = time.time()
    V, _, _, _ = O.lr_potential(u * (1.0 + 0.01 * np.cos(np.arange(grid.shape[2]) * 0.3)), grid,
                                fn, kf2)
    t_map = time.time() - t1
    t2 = time.time()
    for _ in range(nlcg_steps):
        u, _, _ = O.nlcg(u, V, b, phib, grid, fn, Ne, tol=1e-30, max_iter=1)
    t_step = (time.time() - t2) / nlcg_steps
    return t_map, t_step, (grid, b, phib, u)


def cpu_estimate(t_setup, t_forces, t_map, t_step, counts):
    """Oracle seconds per ground state + forces: setup + NLCG steps x (time per step) + kernel
    maps x (time per map) + forces, with the step and map counts of the oracle's own run."""
    nlcg_total, maps = counts
    return t_setup + nlcg_total * t_step + maps * t_map + t_forces


def cpu_sample(cell, budget_s=20.0):
    """The oracle on a bounded sample of the benchmark cell (setup, forces, one kernel map and
    a few NLCG steps, about budget_s of host time), scaled to one ground state + forces with
    the NLCG-step and kernel-map counts of the oracle's own converged run of this cell
    (tests/golden/al108_wt.json)."""
    counts = oracle_counts()
    t0 = time.time()
    state, t_setup, t_forces = cpu_setup(cell)
    t_map, t_step, state = cpu_iteration(cell, state, 1)
    steps = [t_step]
    while time.time() - t0 < budget_s and len(steps) < 6:
        t, state = cpu_nlcg_only(cell, state)
        steps.append(t)
    t_step = statistics.median(steps)
    est = cpu_estimate(t_setup, t_forces, t_map, t_step, counts)
    sample = (f"oracle (numpy FP64, FFT-exact solves, one host core) on the 108-atom 96^3 cell: "
              f"setup {t_setup:.1f} s, forces {t_forces:.1f} s, one kernel map {t_map:.2f} s, "
              f"{len(steps)} NLCG steps at {t_step:.2f} s (median); scaled with the oracle's own "
              f"run of this cell ({counts[0]} NLCG steps, {counts[1]} kernel maps, "
              f"tests/golden/al108_wt.json)")
    return est, sample, time.time() - t0


def _host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _oracle_pool(nproc):
    """A pool of nproc spawned processes (no process inherits the parent's CUDA state), each
    with one numerical-library thread so that the processes fill the cores without
    oversubscribing them."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(nproc)


def _oracle_sample_worker(budget_s):
    from paper_1412_8250_gb300 import workloads as W
    est, _, wall = cpu_sample(W.al108_cell(), budget_s)
    return est, wall


def cpu_sample_all_cores(budget_s=20.0):
    """The bounded oracle sample of cpu_sample in one process per host core at once: each
    process's estimate of one ground state + forces while every core works, and the host's
    throughput, cores / (median estimate), as seconds per ground state.  Returns
    (s per ground state for the host, median per-process estimate, cores, wall seconds)."""
    ncores = _host_cores()
    t0 = time.time()
    with _oracle_pool(ncores) as pool:
        res = pool.map(_oracle_sample_worker, [budget_s] * ncores)
    med = statistics.median(r[0] for r in res)
    return med / ncores, med, ncores, time.time() - t0


def cpu_nlcg_only(cell, state):
    """One NLCG step of the oracle at zero V_LR, timed (a line-search step costs the same
    whatever V_LR is).  Returns (seconds, state)."""
    import numpy as np
    import oracle as O
    grid, b, phib, u = state
    t = time.time()
    u, _, _ = O.nlcg(u, np.zeros(grid.shape), b, phib, grid, O.wt_functional(), cell.n_electrons,
                     tol=1e-30, max_iter=1)
    return time.time() - t, (grid, b, phib, u)


def config1_measured(torch, B, Fn, W):
    """A like-for-like measured pair on the small cell the oracle finishes in seconds: the
    4-atom FCC cell of the TFW configuration (a = 7.6, sigma = 0.7, 32^3, order 12, uniform
    start), one full ground state + forces by the oracle on one host core and by the GPU in
    both forms (after one untimed run)."""
    import numpy as np
    import oracle as O
    cell = W.al4_cell()
    grid = O.Grid(cell.n, cell.L, 6)
    t = time.time()
    ref = O.scf_ground_state(grid, cell.R, cell.Z, cell.sigma, cell.rc, O.tfw_functional(),
                             nlcg_tol=1e-7)
    O.forces(ref.phi, cell.R, cell.Z, cell.sigma, cell.rc, grid)
    t_oracle = time.time() - t
    out = {"workload": "4-atom FCC cell, a=7.6 bohr, Gaussian ions Z=3 sigma=0.7 r_c=7, 32^3, "
                       "12th-order FD, TFW (lambda=1/5) + PZ LDA, ground state + forces",
           "oracle_s": t_oracle, "oracle_cores": 1}
    h = B.of_grid_create(cell.n, cell.L, 6, torch.cuda.current_stream())
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    for name, prec in (("gpu_mixed_s", B.OF_F32), ("gpu_plain_f64_cg_s", B.OF_F64)):
        o = B.of_default_scf_opts()
        o.precision = prec
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        for k in range(2):
            u.fill_(1.0)
            phi.zero_()
            torch.cuda.synchronize()
            t = time.time()
            res = B.of_scf_ground_state(h, sysd, Fn.tfw(), o, u, phi)
            B.of_forces(h, sysd, u, phi)
            torch.cuda.synchronize()
            dt = time.time() - t
        out[name] = dt
        out[name.replace("_s", "_energy_error_vs_oracle_ha_per_atom")] = \
            abs(res.energy - ref.energy) / cell.n_atoms
    B.of_grid_destroy(h)
    out["oracle_over_gpu_mixed"] = t_oracle / out["gpu_mixed_s"]
    return out


def _reference_worker(a):
    """One process of the reference arm: setup and forces (timed once), warm-up NLCG steps, then
    per step one kernel map and one NLCG step, each scaled to a ground state estimate."""
    warmup, steps = a
    from paper_1412_8250_gb300 import workloads as W
    cell = W.al108_cell()
    counts = oracle_counts()
    state, t_setup, t_forces = cpu_setup(cell)
    for _ in range(warmup):
        _, state = cpu_nlcg_only(cell, state)
    vals = []
    for _ in range(steps):
        t_map, t_step, state = cpu_iteration(cell, state, 1)
        vals.append(cpu_estimate(t_setup, t_forces, t_map, t_step, counts))
    return vals


def reference_arm(args, rank, world):
    """The oracle as the reference arm, rank 0 only, on every host core: one spawned process per
    core runs _reference_worker (setup and forces timed once, --warmup NLCG steps, then per step
    one kernel map and one NLCG step of the oracle on the benchmark cell, each scaled to a
    ground state with the oracle's own step counts); a step's value is the host's time per
    ground state, the median of the processes' estimates over the number of processes."""
    if rank != 0:
        return 0
    counts = oracle_counts()
    ncores = _host_cores()
    steps = max(1, args.steps)
    with _oracle_pool(ncores) as pool:
        per_proc = pool.map(_reference_worker, [(args.warmup, steps)] * ncores)
    # step k: the host completes ncores ground states in the median of the processes' estimates
    vals = [statistics.median(p[k] for p in per_proc) / ncores for k in range(steps)]
    v = statistics.median(vals)
    sample = (f"oracle (numpy FP64, FFT-exact solves) on the 108-atom 96^3 cell in {ncores} "
              f"processes at once, one per host core: setup and forces once, then per step one "
              f"kernel map and one NLCG step in every process, each scaled to a ground state with "
              f"the oracle's own run of this cell ({counts[0]} NLCG steps, {counts[1]} kernel "
              f"maps, tests/golden/al108_wt.json); a step's value is the median of the processes' "
              f"estimates over {ncores}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, **WORKLOAD_DETAIL},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def other_configs(torch, B, Fn, W):
    """The other workloads, one timed run each in the chosen form with the benchmark's options
    (their own modes, --config5, --wgc, --relax, --vacancy, add the comparisons): the 3999-atom
    320^3 ground state + forces; the 108-atom ground state + forces with the full WGC functional
    (L = 2); the relaxation of the 108-atom cell; the vacancy formation energy of the perfect
    108-atom cell, unrelaxed and relaxed."""
    import numpy as np
    out = {}
    stream = torch.cuda.current_stream()
    # 3999 atoms, 320^3
    cell = W.al3999_cell()
    h = B.of_grid_create(cell.n, cell.L, 6, stream)
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    _, h0, _, fn, o = make_case(torch, B, Fn, W, "mixed")
    B.of_grid_destroy(h0)
    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    torch.cuda.synchronize()
    t = time.time()
    res = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
    F = B.of_forces(h, sysd, u, phi)
    torch.cuda.synchronize()
    out["large_3999_atoms_320"] = {"s": time.time() - t, "energy_per_atom_ha": res.energy / cell.n_atoms,
                                   "outer_iterations": res.outer_iterations,
                                   "nlcg_steps": res.nlcg_iterations, "fp_error": res.fp_error,
                                   "max_force": float(np.abs(F).max()),
                                   "max_force_sum": float(np.abs(F.sum(0)).max())}
    B.of_grid_destroy(h)
    del u, phi
    # 108 atoms: WGC, relaxation
    cell, h, sysd, fn, o = make_case(torch, B, Fn, W, "mixed")
    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    torch.cuda.synchronize()
    t = time.time()
    res = B.of_scf_ground_state(h, sysd, Fn.wgc(), o, u, phi)
    F = B.of_forces(h, sysd, u, phi)
    torch.cuda.synchronize()
    out["wgc_108_atoms"] = {"s": time.time() - t, "energy_per_atom_ha": res.energy / cell.n_atoms,
                            "outer_iterations": res.outer_iterations, "nlcg_steps": res.nlcg_iterations,
                            "kernel_iterations": res.kernel_iterations, "max_force": float(np.abs(F).max())}
    u.fill_(1.0)
    phi.zero_()
    torch.cuda.synchronize()
    t = time.time()
    R, F, rres = B.of_relax(h, sysd, fn, o, B.of_default_relax_opts(), u, phi, allow=(B.OF_ENOCONV,))
    torch.cuda.synchronize()
    out["relax_108_atoms"] = {"s": time.time() - t, "converged": bool(rres.converged), "steps": rres.steps,
                              "ground_states": rres.evaluations, "max_force": rres.max_force,
                              "energy_per_atom_ha": rres.energy / cell.n_atoms}
    B.of_grid_destroy(h)
    # vacancy formation, perfect 108-atom cell
    pc = W.fcc_supercell((3, 3, 3), points_per_cell=32, sigma=W.SIGMA_LR, rc=W.R_CUT_LR, name="al108_perfect")
    site = int(np.argmin(((pc.R - np.array(pc.L) / 2) ** 2).sum(1)))
    hp = B.of_grid_create(pc.n, pc.L, 6, stream)
    hv = B.of_grid_create(pc.n, B.vacancy_cell_lengths(pc.L, pc.n_atoms), 6, stream)
    psys = B.make_system(pc.R, pc.Z, pc.sigma, pc.rc)
    fields = [torch.ones(pc.shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    HA_EV = 27.211386245988
    for name, ro in (("unrelaxed", None), ("relaxed", B.of_default_relax_opts())):
        fields[0].fill_(1.0)
        fields[2].fill_(1.0)
        fields[1].zero_()
        fields[3].zero_()
        torch.cuda.synchronize()
        t = time.time()
        _, vres = B.of_vacancy_formation(hp, hv, psys, site, fn, o, ro, *fields)
        torch.cuda.synchronize()
        out["vacancy_108_atoms_" + name] = {
            "s": time.time() - t,
            "evf_ev": (vres.evf_unrelaxed if ro is None else vres.evf_relaxed) * HA_EV}
    B.of_grid_destroy(hp)
    B.of_grid_destroy(hv)
    return out


def wgc(args):
    """The 108-atom 96^3 cell with the full WGC functional (L = 2: K_00, K_10 = K_01,
    K_20 = K_02, K_11 of App. A; 16 potentials, 32 shifted solves per kernel map): one ground
    state + forces in the mixed form, timed whole after one untimed ground state; and one
    kernel map V[u] (mixed, tolerance 1e-10) on the GPU against the oracle's map of the same u
    (FFT-exact solves on the host cores).  Prints one JSON line."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    cell, h, sysd, _, o = make_case(torch, B, Fn, W, "mixed")
    fn = Fn.wgc()
    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    times = []
    with ClockSampler(0) as clk:
        for k in range(2):
            u.fill_(1.0)
            phi.zero_()
            torch.cuda.synchronize()
            t = time.time()
            res = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
            F = B.of_forces(h, sysd, u, phi)
            torch.cuda.synchronize()
            times.append(time.time() - t)
        # one kernel map at the ground state, GPU against the oracle
        kf2 = Fn.kf2(cell.n_electrons, cell.L[0] * cell.L[1] * cell.L[2])
        ko = B.of_default_solve_opts()
        ko.precision = B.OF_F32
        vlr = torch.empty_like(u)
        torch.cuda.synchronize()
        t = time.time()
        T_gpu, info = B.of_lr_potential(h, fn, kf2, u, vlr, opts=ko)
        torch.cuda.synchronize()
        t_map_gpu = time.time() - t
    grid = O.Grid(cell.n, cell.L, 6)
    t = time.time()
    V_ref, T_ref, _ = O.lr_potential_wgc(u.cpu().numpy(), grid, O.wgc_functional(), kf2)
    t_map_oracle = time.time() - t
    v_err = float(np.max(np.abs(vlr.cpu().numpy() - V_ref)) / np.max(np.abs(V_ref)))
    line = {"metric": "s per WGC ground state + forces (second-order kernel, 32 shifted solves per map)",
            "value": times[-1], "unit": "s/ground-state", "higher_is_better": False,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("WT-type kernel functional", "full WGC functional (L = 2)")},
            "result": {"energy_per_atom_ha": res.energy / cell.n_atoms, "e_lr_per_atom_ha": res.e_lr / cell.n_atoms,
                       "outer_iterations": res.outer_iterations, "nlcg_steps": res.nlcg_iterations,
                       "poisson_iterations": res.poisson_iterations,
                       "kernel_iterations": res.kernel_iterations, "fp_error": res.fp_error,
                       "max_force": float(np.abs(F).max())},
            "kernel_map": {"gpu_s": t_map_gpu, "gpu_iterations": info.iterations},
            "cpu_baseline": {"value": t_map_oracle, "unit": "s/kernel map", "cores": 1, "kind": "oracle",
                             "sample": "one second-order kernel map V[u] at the GPU ground state, oracle "
                                       "(numpy FP64, FFT-exact solves)",
                             "gpu_vs_oracle": {"T_lr_rel_diff": abs(T_gpu - T_ref) / abs(T_ref),
                                               "V_lr_max_rel_diff": v_err}},
            "times_s": times, "clocks": clk.summary()}
    B.of_grid_destroy(h)
    print(json.dumps(line), flush=True)
    return 0


def relax_case(args):
    """Geometry relaxation (Sec. 3.3) of the 108-atom 96^3 cell from its +-0.1 bohr displaced
    positions, WT-type functional, mixed form, to max |F| < 1e-3 Ha/bohr: every line-search
    point a ground state warm-started from the previous one, plus its forces.  Timed whole;
    prints one JSON line."""
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    cell, h, sysd, fn, o = make_case(torch, B, Fn, W, "mixed")
    ro = B.of_default_relax_opts()
    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t = time.time()
        R, F, res = B.of_relax(h, sysd, fn, o, ro, u, phi, allow=(B.OF_ENOCONV,))
        torch.cuda.synchronize()
        wall = time.time() - t
    line = {"metric": "s per geometry relaxation (NLCG + secant on the forces, max |F| < 1e-3 Ha/bohr)",
            "value": wall, "unit": "s/relaxation", "higher_is_better": False, "dtype": "f64+f32",
            "data": "synthetic", "config": {"workload": WORKLOAD.replace("ground state + forces", "geometry relaxation")},
            "result": {"converged": bool(res.converged), "steps": res.steps, "ground_states": res.evaluations,
                       "s_per_ground_state": wall / max(1, res.evaluations),
                       "energy_per_atom_ha": res.energy / cell.n_atoms, "max_force": res.max_force,
                       "max_displacement_bohr": float(np.abs(R - cell.R).max())},
            "clocks": clk.summary()}
    B.of_grid_destroy(h)
    print(json.dumps(line), flush=True)
    return 0


def convergence_case(args):
    """Sec. 5.1's study on the GPU: ground-state energy and forces of the 4-atom TFW cell with
    the corner atom at (0.80, 0.56, 0.42) for 16..48 points per 7.6 bohr and FD orders 2, 6, 12,
    errors against the order-12 result on 96 points, and the fitted rates.  The reference's own
    error is estimated from the order-12 results on 64 and 96 points (the 64-point error bounds
    it, scaled by (64/96)^11 at the order-12 rate); points whose error is within 100x of that
    estimate (or of 1e-12, the ground state's own rounding floor) are left out of the fits, and
    the floor is reported.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    stream = torch.cuda.current_stream()
    fn = Fn.tfw()

    def run(n, N):
        c = W.al4_displaced_cell(points_per_cell=n)
        h = B.of_grid_create(c.n, c.L, N, stream)
        try:
            o = B.of_default_scf_opts()
            o.nlcg_tol = 1e-10
            u = torch.ones(c.shape, dtype=torch.float64, device="cuda")
            phi = torch.zeros_like(u)
            sysd = B.make_system(c.R, c.Z, c.sigma, c.rc)
            res = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
            F = B.of_forces(h, sysd, u, phi)
        finally:
            B.of_grid_destroy(h)
        return res.energy / c.n_atoms, F

    t0 = time.time()
    E_ref, F_ref = run(96, 6)
    E64, F64 = run(64, 6)
    shrink = (64.0 / 96.0) ** 11
    floor = {"energy_error_ha_per_atom": max(1e-12, abs(E64 - E_ref) * shrink),
             "force_error_ha_per_bohr": max(1e-12, float(np.abs(F64 - F_ref).max()) * shrink)}
    ns = (16, 20, 24, 32, 40, 48)
    out = {}
    for N in (1, 3, 6):
        rows = []
        for n in ns:
            E, F = run(n, N)
            rows.append({"points_per_edge": n, "h_bohr": 7.6 / n,
                         "energy_error_ha_per_atom": abs(E - E_ref),
                         "force_error_ha_per_bohr": float(np.abs(F - F_ref).max())})
        for key in ("energy_error_ha_per_atom", "force_error_ha_per_bohr"):
            e = [r[key] for r in rows]
            ok = [i for i in range(len(ns)) if e[i] > 100.0 * floor[key]]
            rate = (float(np.polyfit(np.log([7.6 / ns[i] for i in ok]), np.log([e[i] for i in ok]), 1)[0])
                    if len(ok) >= 2 else None)
            out.setdefault(f"order_{2 * N}", {})[key.split("_error")[0] + "_rate"] = rate
        out[f"order_{2 * N}"]["rows"] = rows
    line = {"metric": "mesh convergence rates of the energy and forces (Sec. 5.1)", "unit": "rate",
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4-atom FCC Al-like cell, a=7.6 bohr, corner atom at (0.80, 0.56, 0.42), "
                                   "TFW, reference: order 12 on 96 points per edge"},
            "wall_s": time.time() - t0, "result": out,
            "reference_error_estimate": floor,
            "fit_threshold": {k: 100.0 * v for k, v in floor.items()}}
    print(json.dumps(line), flush=True)
    return 0


def vacancy_case(args):
    """Vacancy formation energy (Sec. 5.6) of the perfect 108-atom 3x3x3 FCC cell (a = 7.6,
    96^3, WT-type functional, mixed form, the benchmark's options), the site nearest the centre
    removed and the vacancy cell scaled to the same volume per atom: the two ground states at
    once, then the vacancy cell's relaxation to max |F| < 1e-3 Ha/bohr.  Timed whole; prints one
    JSON line."""
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    _, h0, _, fn, o = make_case(torch, B, Fn, W, "mixed")
    B.of_grid_destroy(h0)
    cell = W.fcc_supercell((3, 3, 3), points_per_cell=32, sigma=W.SIGMA_LR, rc=W.R_CUT_LR,
                           name="al108_perfect")
    site = int(np.argmin(((cell.R - np.array(cell.L) / 2) ** 2).sum(1)))
    stream = torch.cuda.current_stream()
    hp = B.of_grid_create(cell.n, cell.L, 6, stream)
    hv = B.of_grid_create(cell.n, B.vacancy_cell_lengths(cell.L, cell.n_atoms), 6, stream)
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    ro = B.of_default_relax_opts()
    fields = [torch.ones(cell.shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    out = {}
    with ClockSampler(0) as clk:
        for name, r in (("unrelaxed", None), ("relaxed", ro)):
            fields[0].fill_(1.0)
            fields[2].fill_(1.0)
            fields[1].zero_()
            fields[3].zero_()
            torch.cuda.synchronize()
            t = time.time()
            R, res = B.of_vacancy_formation(hp, hv, sysd, site, fn, o, r, *fields)
            torch.cuda.synchronize()
            out[name] = (time.time() - t, R, res)
    HA_EV = 27.211386245988
    tu, _, ru = out["unrelaxed"]
    tr, Rr, rr = out["relaxed"]
    Rv0 = cell.R[np.arange(cell.n_atoms) != site] * (B.vacancy_cell_lengths(cell.L, cell.n_atoms)[0] / cell.L[0])
    line = {"metric": "s per vacancy formation energy (two ground states, then the vacancy cell's relaxation)",
            "value": tr, "unit": "s/vacancy-formation", "higher_is_better": False, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "perfect 108-atom FCC Al-like cell (3x3x3, a=7.6 bohr), centre site removed, "
                                   "vacancy cell scaled to the same volume per atom, 96^3, 12th-order FD, "
                                   "WT-type kernel functional"},
            "result": {"unrelaxed_s": tu, "relaxed_s": tr,
                       "evf_unrelaxed_ev": ru.evf_unrelaxed * HA_EV, "evf_relaxed_ev": rr.evf_relaxed * HA_EV,
                       "e_perfect_per_atom_ha": rr.e_perfect / cell.n_atoms,
                       "relax_steps": rr.relax_steps, "vacancy_ground_states": rr.evaluations,
                       "max_force": rr.max_force,
                       "max_displacement_bohr": float(np.abs(Rr - Rv0).max())},
            "clocks": clk.summary()}
    B.of_grid_destroy(hp)
    B.of_grid_destroy(hv)
    print(json.dumps(line), flush=True)
    return 0


def mixing_study(args):
    """Sec. 5.3 as a benchmark: the 108-atom 96^3 ground state (WT-type, mixed form) with the
    outer fixed point on V_LR (the method) and on u (Table MixComparison's alternative), each
    with Anderson history m and mixing parameter zeta in {(3, 1.0), (3, 0.5), (7, 0.3)}: outer
    iterations, NLCG steps, seconds, energy.  Prints one JSON line."""
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    cell, h, sysd, fn, o = make_case(torch, B, Fn, W, "mixed")
    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    runs = []
    with ClockSampler(0) as clk:
        for fpm, name in ((B.OF_FP_VLR, "V_LR"), (B.OF_FP_U, "u")):
            for m, zeta in ((3, 1.0), (3, 0.5), (7, 0.3)):
                o.fixed_point, o.anderson_m, o.anderson_zeta = fpm, m, zeta
                u.fill_(1.0)
                phi.zero_()
                torch.cuda.synchronize()
                t = time.time()
                res = B.of_scf_ground_state(h, sysd, fn, o, u, phi, allow=(B.OF_ENOCONV,))
                torch.cuda.synchronize()
                runs.append({"fixed_point": name, "m": m, "zeta": zeta, "s": time.time() - t,
                             "converged": bool(res.converged), "outer": res.outer_iterations,
                             "nlcg_steps": res.nlcg_iterations, "fp_error": res.fp_error,
                             "energy_per_atom_ha": res.energy / cell.n_atoms})
    line = {"metric": "outer iterations and s per ground state: fixed point on V_LR vs on u, Anderson m / zeta",
            "unit": "s/ground-state", "higher_is_better": False, "data": "synthetic",
            "config": {"workload": WORKLOAD.replace(", ground state + forces", ", ground state")},
            "runs": runs, "clocks": clk.summary()}
    B.of_grid_destroy(h)
    print(json.dumps(line), flush=True)
    return 0


def config5(args):
    """The 3999-atom cell (10x10x10 FCC minus the centre site, +-0.1 bohr displacements, seed 5),
    320^3 grid (32.8 M points): one ground state + forces in the chosen form (mixed precision,
    the benchmark's options, preconditioned NLCG), timed whole; the same with the paper's plain
    NLCG, timed whole; the plain FP64 CG form timed on bounded samples (the first outer
    iteration stopped after 2 and after 4 NLCG steps, and one FP64 kernel map) and
    extrapolated with the plain-NLCG mixed run's NLCG and outer counts (both run the same
    algorithm).  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    cell = W.al3999_cell()
    stream = torch.cuda.current_stream()
    h = B.of_grid_create(cell.n, cell.L, 6, stream)
    sysd = B.make_system(cell.R, cell.Z, cell.sigma, cell.rc)
    fn = Fn.wt()

    def opts(prec, pshift=0.0):
        o = B.of_default_scf_opts()
        o.precision = prec
        o.fp_tol = 1e-6
        o.anderson_m = 3
        o.anderson_zeta = 1.0
        o.nlcg_tol_rel = 3e-2       # the benchmark's inexact schedule (make_case)
        o.poisson.inner_tol = POISSON_PASS_TOL
        o.nlcg_precond_shift = pshift
        o.nlcg_precond_low = NLCG_PRECOND_LOW if pshift > 0.0 else 0.0
        return o

    u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(u)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t = time.time()
        res = B.of_scf_ground_state(h, sysd, fn, opts(B.OF_F32, NLCG_PRECOND_SHIFT), u, phi)
        F = B.of_forces(h, sysd, u, phi)
        torch.cuda.synchronize()
        t_mixed = time.time() - t
        u_gs = u.clone()
        u.fill_(1.0)
        phi.zero_()
        torch.cuda.synchronize()
        t = time.time()
        res_p = B.of_scf_ground_state(h, sysd, fn, opts(B.OF_F32), u, phi)
        B.of_forces(h, sysd, u, phi)
        torch.cuda.synchronize()
        t_plain_nlcg = time.time() - t
        samples = {}
        for k in (2, 4):
            o = opts(B.OF_F64)
            o.fp_max_iter = 1
            o.nlcg_max_iter = k
            u.fill_(1.0)
            phi.zero_()
            torch.cuda.synchronize()
            t = time.time()
            B.of_scf_ground_state(h, sysd, fn, o, u, phi, allow=(B.OF_ENOCONV,))
            torch.cuda.synchronize()
            samples[k] = time.time() - t
        ko = B.of_default_solve_opts()
        vlr = torch.zeros_like(u)
        kf2 = Fn.kf2(cell.n_electrons, cell.L[0] * cell.L[1] * cell.L[2])
        torch.cuda.synchronize()
        t = time.time()
        B.of_lr_potential(h, fn, kf2, u_gs, vlr, opts=ko)
        torch.cuda.synchronize()
        kmap = time.time() - t
    per_step = (samples[4] - samples[2]) / 2.0
    est = samples[2] + per_step * (res_p.nlcg_iterations - 2) + kmap * (res_p.outer_iterations - 1)
    stencil = stencil_rates(torch, B, cell.shape, cell.L, reps=10)
    line = {"metric": METRIC, "unit": UNIT, "higher_is_better": False, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "3999-atom FCC Al-like cell (10x10x10 minus the centre site, "
                                   "a=7.6 bohr, +-0.1 bohr displacements, seed 5), 320^3, "
                                   "12th-order FD, WT-type kernel (sigma=1.2, r_c=10); ground "
                                   "state + forces"},
            "mixed_multigrid_s": t_mixed,
            "mixed_multigrid_plain_nlcg_s": t_plain_nlcg,
            "plain_nlcg_counts": {"outer_iterations": res_p.outer_iterations,
                                  "nlcg_steps": res_p.nlcg_iterations,
                                  "energy_difference_ha_per_atom":
                                      abs(res_p.energy - res.energy) / cell.n_atoms},
            "plain_fp64_cg_s_estimate": est,
            "plain_fp64_sample": {"first_outer_2_nlcg_steps_s": samples[2],
                                  "first_outer_4_nlcg_steps_s": samples[4],
                                  "per_nlcg_step_s": per_step, "fp64_kernel_map_s": kmap},
            "result": {"energy_ha": res.energy, "energy_per_atom_ha": res.energy / cell.n_atoms,
                       "outer_iterations": res.outer_iterations, "nlcg_steps": res.nlcg_iterations,
                       "poisson_iterations": res.poisson_iterations,
                       "kernel_iterations": res.kernel_iterations, "fp_error": res.fp_error,
                       "max_force": float(np.abs(F).max()),
                       "force_sum": [float(x) for x in F.sum(0)],
                       "u_min": float(u_gs.min())},
            "stencil_320": stencil, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    B.of_grid_destroy(h)
    return 0


def whole_job_value(step_ms, steps, world, device="cuda"):
    """Replicas: every rank solves its own copy of the cell, so the job's time is the slowest
    rank's (max over ranks) and the job completes world x steps ground states in it.  Returns
    (job milliseconds, seconds per ground state of the whole job)."""
    total_ms = float(sum(step_ms))
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / 1e3 / (steps * world)


def batched_ground_states(torch, B, Fn, W, ncells):
    """Ground states + forces of the first ncells cells of the 64-cell set (reps 2..4 per axis,
    64-128 points per axis, half with a vacancy, +-0.1 bohr, seed 3; WT-type kernel, the
    benchmark's options): one batched call (each cell's solver on its own stream of a pool,
    driven by its own host thread) against the same ground states one after another.  An
    untimed batched call cut short (one outer iteration of three NLCG steps) first creates
    every cell's workspace, multigrid hierarchy and graphs."""
    cells = W.batched_cells()[:ncells]
    stream = torch.cuda.current_stream()
    grids = [B.of_grid_create(c.n, c.L, 6, stream) for c in cells]
    systems = [B.make_system(c.R, c.Z, c.sigma, c.rc) for c in cells]
    _, h0, _, _, o = make_case(torch, B, Fn, W, "mixed")
    B.of_grid_destroy(h0)
    fn = Fn.wt()
    us = [torch.ones(c.shape, dtype=torch.float64, device="cuda") for c in cells]
    phis = [torch.zeros_like(x) for x in us]

    def batched(opts, allow=()):
        for x, p in zip(us, phis):
            x.fill_(1.0)
            p.zero_()
        r = B.of_scf_ground_state_batched(grids, systems, fn, opts, us, phis, allow=allow)
        forces = [B.of_forces(g, s, x, p) for g, s, x, p in zip(grids, systems, us, phis)]
        return r, forces

    def sequential():
        out = []
        for g, s, x, p in zip(grids, systems, us, phis):
            x.fill_(1.0)
            p.zero_()
            out.append(B.of_scf_ground_state(g, s, fn, o, x, p))
            B.of_forces(g, s, x, p)
        return out

    short = B.of_scf_opts.from_buffer_copy(o)
    short.fp_max_iter, short.nlcg_max_iter = 1, 3
    batched(short, allow=(B.OF_ENOCONV,))
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t = time.time()
        rb, _ = batched(o)
        torch.cuda.synchronize()
        tb = time.time() - t
        t = time.time()
        rs = sequential()
        torch.cuda.synchronize()
        ts = time.time() - t
    de = max(abs(a.energy - b.energy) / c.n_atoms for a, b, c in zip(rb, rs, cells))
    out = {"workload": f"first {len(cells)} cells of the 64-cell set (seed 3), WT-type kernel, "
                       "ground state + forces each",
           "cells": len(cells), "points": int(sum(c.n_points for c in cells)),
           "atoms": int(sum(c.n_atoms for c in cells)),
           "batched_s": tb, "sequential_s": ts, "speedup": ts / tb,
           "all_converged": all(r.converged for r in rb),
           "max_energy_difference_ha_per_atom": de,
           "energies_per_atom_ha": [r.energy / c.n_atoms for r, c in zip(rb, cells)],
           "clocks": clk.summary()}
    for g in grids:
        B.of_grid_destroy(g)
    return out


def config3(args):
    """--config3: the batched ground states of the first --cells cells as one JSON line."""
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    r = batched_ground_states(torch, B, Fn, W, args.cells)
    line = {"metric": "s per batch of ground states + forces", "unit": "s", "higher_is_better": False,
            "data": "synthetic", "config": {"workload": r["workload"], "points": r["points"],
                                            "atoms": r["atoms"]}, **r}
    print(json.dumps(line), flush=True)
    return 0


def kernel_case(args):
    """Bounded pieces of the benchmark step, for profiler captures."""
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W
    B.load()
    if args.kernel_case == "net160":
        # three applications of the preconditioner network on a 160^3 grid (seeded weights)
        n = 160
        h = B.of_grid_create((n, n, n), (0.2375 * n,) * 3, 6, torch.cuda.current_stream())
        net = B.of_precond_create(W.initial_network(0))
        r = torch.from_numpy(W.random_field((n, n, n), seed=1).astype(np.float32)).cuda()
        z = torch.empty_like(r)
        for _ in range(3):
            B.of_precond_apply(h, net, r, z)
        torch.cuda.synchronize()
        B.of_precond_destroy(net)
        B.of_grid_destroy(h)
        return 0
    if args.kernel_case in ("stencil96", "stencil320"):
        n = 96 if args.kernel_case == "stencil96" else 320
        h = B.of_grid_create((n, n, n), (0.2375 * n,) * 3, 6, torch.cuda.current_stream())
        for dt, tdt in [(B.OF_F32, torch.float32), (B.OF_F64, torch.float64)]:
            x = torch.rand((n, n, n), dtype=tdt, device="cuda")
            y = torch.empty_like(x)
            for _ in range(3):
                B.of_laplacian_apply(h, dt, x, y)
        torch.cuda.synchronize()
        B.of_grid_destroy(h)
        return 0
    cell, h, sysd, fn, o = make_case(torch, B, Fn, W, args.precision)
    if args.kernel_case == "scf96_short":
        # the benchmark's ground state cut short (2 outer iterations of at most 10 NLCG steps):
        # every kernel class of the step, in a launch count a profiler can list
        o.fp_max_iter = 2
        o.nlcg_max_iter = 10
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        B.of_scf_ground_state(h, sysd, fn, o, u, phi, allow=(B.OF_ENOCONV,))
        B.of_forces(h, sysd, u, phi)
        torch.cuda.synchronize()
        B.of_grid_destroy(h)
        return 0
    if args.kernel_case == "poisson96":
        rho = torch.from_numpy(W.random_field(cell.shape, seed=3, kind="smooth")).cuda()
        so = B.of_default_solve_opts()
        so.precision = o.precision
        for _ in range(4):
            phi = torch.zeros_like(rho)
            B.of_poisson_solve(h, rho, phi, so)
    else:
        u = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
        phi = torch.zeros_like(u)
        B.of_scf_ground_state(h, sysd, fn, o, u, phi)
        B.of_forces(h, sysd, u, phi)
    torch.cuda.synchronize()
    B.of_grid_destroy(h)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.kernel_case:
        return kernel_case(args)
    if args.wgc:
        return wgc(args)
    if args.relax:
        return relax_case(args)
    if args.convergence:
        return convergence_case(args)
    if args.vacancy:
        return vacancy_case(args)
    if args.mixing_study:
        return mixing_study(args)
    if args.config5:
        return config5(args)
    if args.config3:
        return config3(args)
    import numpy as np
    import torch
    from paper_1412_8250_gb300 import binding as B, functionals as Fn, workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.load()
    cell, h, sysd, fn, o = make_case(torch, B, Fn, W, args.precision)
    u0 = torch.ones(cell.shape, dtype=torch.float64, device="cuda")
    u = torch.empty_like(u0)
    phi = torch.zeros_like(u0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        res, F = run_step(B, h, sysd, fn, o, u, phi, u0)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    step_ms = []
    launches0 = B.of_launch_count()
    B.of_profile_enable(h, 4)
    barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            res, F = run_step(B, h, sysd, fn, o, u, phi, u0)
            e1.record()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        barrier()
    launches = B.of_launch_count() - launches0
    prof = B.of_profile_read(h)
    B.of_profile_enable(h, 0)
    total_ms, value = whole_job_value(step_ms, args.steps, world, "cuda")

    # end-to-end through the C ABI with host buffers: initial field in, u and phi out
    u_host = torch.ones(cell.shape, dtype=torch.float64).pin_memory()
    out_u = torch.empty(cell.shape, dtype=torch.float64).pin_memory()
    out_phi = torch.empty(cell.shape, dtype=torch.float64).pin_memory()
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t = time.time()
    u.copy_(u_host, non_blocking=True)
    res_e2e = B.of_scf_ground_state(h, sysd, fn, o, u, phi)
    F_e2e = B.of_forces(h, sysd, u, phi)
    out_u.copy_(u, non_blocking=True)
    out_phi.copy_(phi, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.time() - t
    h2d = u_host.numel() * 8
    d2h = 2 * out_u.numel() * 8 + F_e2e.size * 8

    stencil = stencil_rates(torch, B, cell.shape, cell.L)
    stencil320 = None if rank != 0 else stencil_rates(torch, B, (320, 320, 320), (76.0, 76.0, 76.0),
                                                      reps=20)
    batched = None if (args.no_batched or rank != 0) else batched_compare(torch, B, W)
    batched_gs = None if (args.no_batched or rank != 0) else batched_ground_states(torch, B, Fn, W, 64)
    learned = None if (args.no_learned or rank != 0) else learned_compare(torch, B, W)
    others = None if (args.no_other_configs or rank != 0) else other_configs(torch, B, Fn, W)
    compare = None
    if not args.no_compare_f64 and rank == 0:
        # the plain FP64 CG / COCG form with the same options (the chosen form's counterpart),
        # one ground state + forces timed whole
        _, h64, s64, fn64, o64 = make_case(torch, B, Fn, W, "f64")
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.time()
        u.copy_(u0)
        r64 = B.of_scf_ground_state(h64, s64, fn64, o64, u, phi)
        F64 = B.of_forces(h64, s64, u, phi)
        torch.cuda.synchronize()
        t64 = time.time() - t
        # the chosen form without the NLCG preconditioner (the paper's plain NLCG): what the
        # preconditioner alone gains
        o_plain_nlcg = B.of_scf_opts.from_buffer_copy(o)
        o_plain_nlcg.nlcg_precond_shift = 0.0
        o_plain_nlcg.nlcg_precond_low = 0.0
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.time()
        u.copy_(u0)
        rpn = B.of_scf_ground_state(h, sysd, fn, o_plain_nlcg, u, phi)
        B.of_forces(h, sysd, u, phi)
        torch.cuda.synchronize()
        t_pn = time.time() - t
        compare = {"plain_fp64_cg_s_per_ground_state": t64,
                   "chosen_with_plain_nlcg_s_per_ground_state": t_pn,
                   "chosen_with_plain_nlcg_nlcg_steps": rpn.nlcg_iterations,
                   "chosen_s_per_ground_state": value,
                   "speedup_chosen_vs_plain_fp64": t64 / value,
                   "energy_difference_ha_per_atom": abs(r64.energy - res.energy) / cell.n_atoms,
                   "max_force_difference_ha_per_bohr": float(np.max(np.abs(F64 - F))),
                   "plain_fp64": {"outer_iterations": r64.outer_iterations,
                                  "nlcg_steps": r64.nlcg_iterations,
                                  "poisson_iterations": r64.poisson_iterations,
                                  "kernel_iterations": r64.kernel_iterations},
                   "plain_fp64_vs_oracle": errors_vs_oracle(r64, F64, cell.n_atoms)}
        B.of_grid_destroy(h64)
    config1 = None if (rank != 0 or world > 1 or args.no_cpu_baseline) else \
        config1_measured(torch, B, Fn, W)

    # roofline of the dominant kernel class (largest extrapolated time in the timed region)
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda p: p["mean_ms"] * p["launches"]) if prof else None
    roofline = None
    if dom and dom["mean_ms"] > 0:
        achieved = dom["bytes_per_launch"] / (dom["mean_ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None, "kernel": dom["kernel"],
                    "peak_kind": peak_kind,
                    "launches": dom["launches"], "mean_us": dom["mean_ms"] * 1e3,
                    "bytes_per_launch": dom["bytes_per_launch"],
                    "bytes_model": "every field a fused sweep reads or writes, once per point of "
                                   "its level (CG iteration 10 words, Chebyshev step 6, residual "
                                   "3, transfers 1-2 per fine point), halos not counted"}
        if dom["kernel"] in ("mg_pcg_pass_graph", "mg_cocg_pass_graph") and prof:
            # the same time against the Krylov iterations' own bytes only (10 words per point
            # per iteration: FP32 for CG, complex FP32 for COCG), the V-cycle's sweeps left out
            cocg = dom["kernel"] == "mg_cocg_pass_graph"
            passes = sum(p["launches"] for p in prof if p["kernel"] == dom["kernel"])
            its = (res.kernel_iterations if cocg else res.poisson_iterations) * args.steps / max(1, passes)
            cg_bytes = its * (80.0 if cocg else 40.0) * cell.n_points
            roofline["cg_iterations_per_launch"] = its
            roofline["frac_cg_bytes_only"] = cg_bytes / (dom["mean_ms"] * 1e-3) / 1e9 / peak
            if cocg and cell.n_points == 96 ** 3:
                roofline["traffic"] = its * COCG96_DRAM_BYTES_PER_ITERATION
                roofline["traffic_note"] = (
                    "ncu dram__bytes_read.sum + dram__bytes_write.sum of the pass's kernels "
                    "launched one by one from a cold L2 (OF_NO_GRAPHS=1, 28 iterations of the "
                    "first kernel map: 167 MB per V-cycle + COCG iteration), scaled by the "
                    "iterations per pass; inside the graphs the fields stay in L2")
            roofline["note"] = ("latency-bound: at 96^3 every field stays in L2 and one "
                                "preconditioned iteration is a chain of ~17 dependent launches"
                                + ("; up to four shifted systems are solved at once (a chain of "
                                   "twin handles), so a pass's events also span the passes "
                                   "beside it and its mean duration overstates its own time"
                                   if cocg else ""))
    roofline_320 = roofline_320_f64 = alu = None
    if stencil320:
        roofline_320 = {"kernel": "stencil2_kernel (of_laplacian_apply, FP32, order 12, 320^3)",
                        "bound": "hbm", "achieved": stencil320["f32"]["gbs"], "peak": peak,
                        "unit": "GB/s", "frac": stencil320["f32"]["gbs"] / peak,
                        "traffic": STENCIL320_DRAM_BYTES, "bytes_per_launch": 8.0 * 320 ** 3,
                        "peak_kind": peak_kind}
        # the FP64 sweep (the refinement residuals) is bound by FP64 arithmetic, not by HBM:
        # its roofline is the measured DFMA rate of this GPU
        alu = alu_peaks(B, torch)
        achieved = stencil320["f64"]["gpts"] * 1e9 * STENCIL_F64_FLOPS_PER_POINT
        roofline_320_f64 = {"kernel": "stencil_kernel<double> (of_laplacian_apply, FP64, order "
                                      "12, 320^3)",
                            "bound": "alu", "achieved": achieved / 1e12,
                            "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                            "frac": achieved / 1e12 / alu["fp64_tflops"], "traffic": None,
                            "flops_per_point": STENCIL_F64_FLOPS_PER_POINT,
                            "peak_kind": "measured (of_alu_peak: DFMA chains on every SM, this run)"}

    clocks = clk.summary()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host_s, per_proc, ncores, wall = cpu_sample_all_cores()
        counts = oracle_counts()
        sample = (f"oracle (numpy FP64, FFT-exact solves) on the 108-atom 96^3 cell in {ncores} "
                  f"processes at once, one per host core: each times setup, forces, one kernel "
                  f"map and up to 6 NLCG steps (~20 s) and scales them with the oracle's own run "
                  f"of this cell ({counts[0]} NLCG steps, {counts[1]} kernel maps, "
                  f"tests/golden/al108_wt.json) to {per_proc:.0f} s per ground state (median over "
                  f"the processes); the host completes {ncores} ground states in that time")
        cpu = {"value": host_s, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
               "per_core_s": per_proc, "wall_s": wall, "measured_small_cell": config1}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, **WORKLOAD_DETAIL, "form": args.precision,
                           "l2": "flushed between steps (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "roofline": roofline, "roofline_stencil_320": roofline_320,
                "roofline_stencil_320_f64": roofline_320_f64, "alu_peaks": alu,
                "cpu_baseline": cpu, "clocks": clocks,
                "stencil_96": stencil, "stencil_320": stencil320,
                "result": {"energy_ha": res.energy, "energy_per_atom_ha": res.energy / cell.n_atoms,
                           "outer_iterations": res.outer_iterations,
                           "nlcg_steps": res.nlcg_iterations,
                           "poisson_iterations": res.poisson_iterations,
                           "kernel_iterations": res.kernel_iterations,
                           "fp_error": res.fp_error, "max_force": float(np.abs(F).max()),
                           **(errors_vs_oracle(res, F, cell.n_atoms) or {})},
                "kernel_profile": prof, "step_ms": step_ms, "batched_poisson_64_cells": batched,
                "batched_ground_states_64": batched_gs,
                "learned_preconditioner": learned, "other_workloads": others}
        if compare:
            line["compare"] = compare
        print(json.dumps(line), flush=True)
    B.of_grid_destroy(h)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
