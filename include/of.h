/*
 * of.h -- C ABI of the GB300 library for periodic orbital-free DFT with higher-order finite
 * differences (Ghosh & Suryanarayana, arXiv:1412.8250).
 *
 * Conventions for every entry point:
 *  - A field on the n1 x n2 x n3 grid is an array of n1*n2*n3 values, x fastest:
 *    f[i + n1*(j + n2*k)] is the value at x = (i h1, j h2, k h3), h_d = L_d / n_d (Sec. 4).
 *  - Complex fields are interleaved (re, im) pairs of doubles, 2*n1*n2*n3 doubles.
 *  - Field pointers are DEVICE pointers owned by the caller; the library never frees them.
 *    Atom data (of_system), coefficient arrays and force outputs are HOST pointers.
 *  - All device work is enqueued on the stream given to of_grid_create.  Calls that return
 *    host scalars (energies, iteration counts, forces) synchronise that stream before
 *    returning; the others are asynchronous.
 *  - Atomic units throughout (bohr, hartree).
 *  - Errors: every call returns an of_status; on failure of_last_error() gives a message
 *    (thread-local).  No C++ exception crosses this boundary.  A solver that stops at its
 *    iteration limit returns OF_ENOCONV with its best iterate written to the output.
 *  - A grid handle holds device workspace (allocated at create and on the first call that
 *    needs more) and is used by one host thread at a time.
 */
#ifndef OF_H
#define OF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OF_OK = 0,
    OF_EINVAL = 1,       /* invalid argument (null pointer, size, unsupported order) */
    OF_ENOMEM = 2,       /* device or host allocation failed */
    OF_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    OF_ENOCONV = 4,      /* iteration limit reached before the tolerance */
    OF_EBREAKDOWN = 5,   /* Krylov breakdown (zero curvature / zero bilinear form) */
    OF_ETIMEOUT = 6      /* a bounded device wait gave up */
} of_status;

typedef enum {
    OF_F64 = 0,          /* plain FP64 */
    OF_F32 = 1           /* FP32 sweeps; in solvers: FP32 inner Krylov + FP64 refinement */
} of_dtype;

/* Line search of the NLCG step (App. C).  OF_LINE_BRENT: Brent's method on the energy, as in
 * the paper (Sec. 3.3).  OF_LINE_SLOPE (default): the root of dE/ds by a safeguarded secant,
 * E and dE/ds from one pass over the grid; the same minimiser in about a third of the passes. */
typedef enum {
    OF_LINE_BRENT = 0,
    OF_LINE_SLOPE = 1
} of_line_search;

/* Discrete form of the reported vW energy (of_scf_opts.vw_energy). */
typedef enum {
    OF_VW_LAPLACIAN = 0,
    OF_VW_GRADIENT = 1
} of_vw_energy;

/* Variable of the outer fixed point with Anderson mixing (App. D). */
typedef enum {
    OF_FP_VLR = 0,
    OF_FP_U = 1
} of_fixed_point;

typedef struct of_grid of_grid;
typedef struct of_precond of_precond;   /* learned preconditioner (of_precond_create) */

/* Krylov solve options.  tol is the target of the true FP64 relative residual
 * ||b - A x|| / ||b||.  precision OF_F64: CG/COCG entirely in FP64.  OF_F32: iterative
 * refinement -- FP64 residual, FP32 Krylov solve of the correction to inner_tol (or only to
 * half of what the solve still needs, when that is less), FP64 update -- repeated until tol;
 * the FP32 Poisson CG is preconditioned by a multigrid
 * V-cycle unless no_multigrid is set, or by the learned network when precond is set (see
 * of_precond_create).  Zero fields take defaults (tol 1e-10, max_iter 20000, inner_tol 1e-5,
 * check_every 8, precond_theta 0.3). */
typedef struct {
    double tol;
    int max_iter;
    int precision;
    double inner_tol;
    int check_every;
    int no_multigrid;      /* 1: plain FP32 CG inner solve for Poisson (no V-cycle) */
    of_precond* precond;   /* non-NULL with OF_F32, in place of the V-cycle: the FP32 inner
                              solve is flexible CG preconditioned by this network (Poisson),
                              or flexible GMRES(8) preconditioned by a few flexible-CG steps
                              with this network on -L_h + kf2 |Q|, applied to the real and
                              imaginary parts of each Arnoldi vector (shifted kernel systems;
                              train the network for that shift, of_precond_set_shift) */
    double precond_theta;  /* a network direction z is kept when cos(r, z) > theta, else the
                              (inner) flexible-CG step is the plain CG step; default 0.3 */
} of_solve_opts;

typedef struct {
    int iterations;        /* Krylov iterations (all passes) */
    int refinements;       /* FP64 residual evaluations */
    double rel_residual;   /* final true FP64 relative residual */
    int net_steps;         /* flexible-CG steps that took the learned network's direction */
} of_solve_info;

/* Ions: positions R[3*M] (x, y, z per ion, bohr), charges Z[M]; each carries the Gaussian
 * charge density b_J(r) = -Z_J (2 pi sigma^2)^{-3/2} exp(-r^2 / (2 sigma^2)) for r <= rc,
 * the stand-in for the pseudopotential charge of Sec. 3.2.  Host pointers. */
typedef struct {
    int n_atoms;
    const double* R;
    const double* Z;
    double sigma;
    double rc;
    int b_from_potential;   /* 0: b_J sampled from its closed form; 1: b_J = -(1/4 pi) L_h V_J,
                               the paper's construction from the potential (Sec. 4), V_J sampled
                               on each ion's box widened by N points (the self energy with it;
                               forces keep the closed-form gradient of b_J) */
    double sigma_ref;       /* overlap correction E_c^* and f^c (App. B): 0 = point reference
                               charges, the closed form 1/2 sum Z_I Z_J erfc(R/2 sigma)/R;
                               > 0 = evaluated on the grid (Eq. RepulsiveCorrection2) with
                               Gaussian reference charges of this width within rc_ref, V_c from
                               one periodic Poisson solve (needs b_from_potential = 0) */
    double rc_ref;          /* cutoff of the reference charges (used when sigma_ref > 0) */
} of_system;

/* Kinetic functional T_TF + lambda T_vW + mu T_LR (Eq. KineticEnergyComponents).  The
 * kernel term (mu != 0) is Eq. LR:KineticEnergy:Linearized with exponents alpha, beta and
 * n_terms rational terms per kernel K_mn (Sec. 3.1, App. A; coefficients interleaved re/im,
 * terms (0,1), (2,3), ... complex-conjugate pairs).  L = 0: the density-independent
 * m = n = 0 term only (P, Q fit K_00).  L = 2 (WGC): the second-order expansion about
 * rho_bar = N_e / Omega, every (m, n) with m + n <= 2: K_00 (P, Q), K_10 = K_01 (P10, Q10),
 * K_20 = K_02 (P20, Q20), K_11 (P11, Q11). */
typedef struct {
    double lambda;
    double mu;
    double alpha;
    double beta;
    int n_terms;
    double P[16];
    double Q[16];
    int L;
    double P10[16], Q10[16];
    double P20[16], Q20[16];
    double P11[16], Q11[16];
} of_functional;

typedef struct {
    double nlcg_tol;        /* normalised residual ||r|| / sqrt(N_e) (App. C); default 1e-7 */
    int nlcg_max_iter;      /* per inner minimisation; default 5000 */
    int nlcg_restart;       /* N_restart; default 50 */
    double fp_tol;          /* fixed-point error ||f_k|| / ||V^_k|| (Sec. 5.3); default 1e-7 */
    int fp_max_iter;        /* default 60 */
    int anderson_m;         /* mixing history m (App. D); default 7 */
    double anderson_zeta;   /* mixing parameter zeta; default 0.3 */
    int precision;          /* OF_F64 plain, or OF_F32 mixed (Poisson and kernel solves) */
    of_solve_opts poisson;  /* defaults: tol 1e-10 */
    of_solve_opts kernel;   /* defaults: tol 1e-10 */
    int verbose;            /* 1: one line per outer iteration on stderr */
    double line_tol;        /* line-search tolerance, relative in the step length (for
                               OF_LINE_SLOPE: |dE/ds| <= line_tol |dE/ds(0)|); default 1e-3 */
    double nlcg_tol_rel;    /* > 0: inexact inner solves, outer step k stops its NLCG at
                               max(nlcg_tol, nlcg_tol_rel * fixed-point error of step k-1);
                               0 (default): every inner solve to nlcg_tol */
    int line_search;        /* of_line_search; default OF_LINE_SLOPE */
    int fixed_point;        /* OF_FP_VLR (default, Sec. 3.3.1): mix V_LR; OF_FP_U: mix u, the
                               alternative of Sec. 5.3 (Table MixComparison) */
    int vw_energy;          /* reported vW energy: OF_VW_LAPLACIAN (default) -(lambda/2) <u, L_h u>,
                               whose gradient is the Hamiltonian's; OF_VW_GRADIENT (lambda/2)
                               int |grad_h u|^2 with the order-2N gradient (Eq.
                               gradient:approximate).  The minimisation is the same. */
    double nlcg_precond_shift;  /* > 0: the NLCG direction is preconditioned by one multigrid
                               V-cycle of -L_h + shift (bohr^-2) applied to the gradient, with the
                               Polak-Ribiere update in its preconditioned form: the real-space
                               preconditioner for Algorithm NLCG that Sec. 5.5 calls for.  Needs a
                               grid the multigrid can coarsen (else ignored).  0 (default): the
                               plain NLCG of App. C */
    double nlcg_precond_low;    /* > 0 with nlcg_precond_shift > 0: the two-shift form
                               (-L_h + low)(-L_h + shift)^{-2}, two V-cycles and one FP32 sweep,
                               which follows the energy's curvature at both ends of the spectrum:
                               ~k^2 at large wave numbers (vW), ~1/k^2 at small ones (Hartree).
                               0 (default): the one-shift form */
} of_scf_opts;

typedef struct {
    double energy;          /* Eq. GroundStateEnergy */
    double e_tf, e_vw, e_lr, e_xc, e_es, e_self, e_corr;
    double fp_error;
    double nlcg_residual;
    int outer_iterations;
    int nlcg_iterations;    /* summed over outer iterations */
    int poisson_iterations;
    int kernel_iterations;
    int line_evaluations;
    int converged;
} of_scf_result;

/* Fill defaults.  Always succeed. */
void of_default_solve_opts(of_solve_opts* o);
void of_default_scf_opts(of_scf_opts* o);

/* Uniform periodic grid of Sec. 4: n_d points of spacing h_d = L_d / n_d per axis, finite
 * differences of order 2N with N = fd_half_order in {1, 3, 6}.  stream is a cudaStream_t
 * (NULL = legacy default stream); the device is the current CUDA device.  Allocates the
 * base workspace.  OF_EINVAL for n_d < 1, L_d <= 0, unsupported N, null out. */
of_status of_grid_create(int n1, int n2, int n3, double L1, double L2, double L3,
                         int fd_half_order, void* stream, of_grid** out);
of_status of_grid_destroy(of_grid* g);

/* y = L_h x: the order-2N central-difference Laplacian of Eq. FD:Laplacian, indices wrapped
 * periodically (Sec. 4).  dtype OF_F64: x, y are double*; OF_F32: float*.  x != y. */
of_status of_laplacian_apply(of_grid* g, of_dtype dtype, const void* x, void* y);

/* Periodic Poisson problem of Eq. Poisson: -(1/4pi) L_h phi = rho, solved by CG on the
 * mean-free part of rho; phi returns with zero mean (Sec. 4).  phi: in = initial guess,
 * out = solution.  rho and phi are double*, n points. */
of_status of_poisson_solve(of_grid* g, const double* rho, double* phi,
                           const of_solve_opts* opts, of_solve_info* info);

/* Shifted solves of Eqs. Helmholtz:beta / Helmholtz:alpha:
 *   -(1/kf2) L_h W_s + Q_s W_s = P_s f,   s = 0 .. nshift-1,
 * by COCG (complex symmetric CG).  f: real double* (n); P, Q: host double[2*nshift]
 * (re, im); W: device complex, nshift consecutive fields of 2n doubles, in = guess,
 * out = solution.  info (optional) sums over the shifts. */
of_status of_kernel_solve(of_grid* g, const double* f, int nshift, const double* P,
                          const double* Q, double kf2, double* W, const of_solve_opts* opts,
                          of_solve_info* info);

/* The Poisson solve of of_poisson_solve (FP64 CG only) for callers that cannot allocate
 * device memory -- code running under an allocator it does not control, or with all device
 * memory reserved up front -- and so cannot create a grid handle.  The paper has no
 * counterpart: this is an interface for such callers.  The grid is passed directly
 * (sizes, side lengths, fd_half_order in {1, 3, 6}, a cudaStream_t or NULL).  rho: device
 * double*, n points; phi: device double*, in = guess, out = mean-free solution.  opts may be
 * NULL (defaults); opts->precision must be OF_F64.
 * This call allocates nothing: its Krylov vectors and reduction scratch live in one static
 * device array of about 10.6 MB that every GPU loading the library holds until exit, which
 * limits the grid to n1*n2*n3 <= 262144 points (OF_EINVAL beyond).  All calls share that array,
 * so calls whose GPU work overlaps (on different streams or threads) race; serialise them.
 * Nor does it create streams, events or CUDA graphs: every CG iteration is launched directly.
 * The first call on a device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  Every call reads solver
 * scalars back to the host, synchronising the stream, at each convergence check and before
 * returning. */
of_status of_poisson_solve_noalloc(int n1, int n2, int n3, double L1, double L2, double L3,
                                   int fd_half_order, void* stream, const double* rho,
                                   double* phi, const of_solve_opts* opts, of_solve_info* info);

/* Poisson solves (as of_poisson_solve) of ncells independent cells at once: grids[c] with
 * rho[c] and phi[c] (device double*, in = guess, out = mean-free solution).  All grids must
 * share the stream and the finite-difference order.  Two forms:
 *  - opts->no_multigrid = 1 (or OF_F64): every Krylov phase of all cells is one grouped launch
 *    and the lockstep FP32 CG iterations (FP64 refinement as in the OF_F32 mode) are replayed
 *    from one CUDA graph; the z extent of the stencil blocks is chosen per set of grid shapes
 *    by timing candidates on the first call.
 *  - OF_F32 with multigrid (the default no_multigrid = 0, every cell coarsenable): each cell
 *    runs the multigrid-preconditioned solve of of_poisson_solve, the cells spread over up to 8
 *    internal streams driven by host threads so that their kernels overlap; the call orders
 *    them after the work queued on the shared stream and the shared stream after them.  The
 *    grids must not be used by other threads meanwhile.
 * infos (optional) receives one record per cell.  Synchronises the stream. */
of_status of_poisson_solve_batched(int ncells, of_grid* const* grids, const double* const* rho,
                                   double* const* phi, const of_solve_opts* opts,
                                   of_solve_info* infos);

/* b = sum over ions and periodic images of b_J (Sec. 3.2) on the grid (device double*),
 * and the self-energy term -(1/2) sum_J int b_J V_J (host double, may be NULL). */
of_status of_pseudocharge(of_grid* g, const of_system* sys, double* b, double* e_self);

/* H u = -(lambda/2) L_h u + (V_TF + mu V_LR + V_xc + phi) u (Eq. EulerLagrange).
 * vlr may be NULL when mu == 0.  All device double*. */
of_status of_hamiltonian_apply(of_grid* g, const of_functional* fn, const double* u,
                               const double* phi, const double* vlr, double* hu);

/* The kernel map V[u] of Eq. MVF (Eq. VLinearResponse:local and the T_LR expression after
 * it).  L = 0: builds f = -(1/kf2) L_h u^{2e} for e = alpha, beta and solves the n_terms
 * shifted systems of each (conjugate pairs solved once).  L = 2: the 16 potentials K_mn *
 * u^{2(k+e)} the second-order sum needs (k <= 2; the right-hand side is the density power
 * itself for (m, n) != (0, 0)), n_terms / 2 shifted solves each, then the sum over m, n, p, q
 * with C_mnpq of Sec. 2.  Writes V_LR (device double*) and T_LR (host double, may be NULL).
 * n_terms must be even.  W_ws: device workspace and warm start of
 * of_lr_workspace_fields(fn) complex fields; NULL uses the handle's own workspace with a
 * zero start. */
int of_lr_workspace_fields(const of_functional* fn);
of_status of_lr_potential(of_grid* g, const of_functional* fn, double kf2, const double* u,
                          double* vlr, double* t_lr, double* W_ws, const of_solve_opts* opts,
                          of_solve_info* info);

/* Ground state (Sec. 3.3.1): fixed point V_LR = V[U(V_LR)] with Anderson mixing (App. D),
 * U by the constrained NLCG of App. C.  u: device double*, in = initial guess (any positive
 * field; it is normalised to N_e = sum Z), out = ground state sqrt(rho).  phi: device
 * double*, out = electrostatic potential.  The energy and its terms go to res. */
of_status of_scf_ground_state(of_grid* g, const of_system* sys, const of_functional* fn,
                              const of_scf_opts* opts, double* u, double* phi,
                              of_scf_result* res);

/* Geometry relaxation (Sec. 3.3): non-linear CG on the nuclear positions with the
 * Polak-Ribiere update (restart at beta < 0 or when the direction is not downhill) and a
 * secant line search on E'(s) = -F(R + s d) . d, started from E'(0) and a trial step that moves
 * the farthest atom by step0 bohr, stopped at |E'(s)| <= line_tol |E'(0)| or after max_line
 * points (the last point is accepted).  Every evaluation is a ground state
 * (of_scf_ground_state with scf, warm-started from the previous evaluation's u) and its forces
 * (of_forces).  Stops when max_J |F_J| < ftol. */
typedef struct {
    double ftol;       /* Ha/bohr; default 1e-3 */
    int max_steps;     /* default 40 */
    double step0;      /* bohr; default 0.05 */
    double line_tol;   /* default 0.1 */
    int max_line;      /* secant points per step; default 4 */
} of_relax_opts;

typedef struct {
    double energy;      /* ground-state energy at the final positions */
    double max_force;   /* max_J |F_J| there */
    int steps;          /* NLCG steps taken */
    int evaluations;    /* ground states (each with forces) computed */
    int converged;      /* max_force < ftol */
} of_relax_result;

void of_default_relax_opts(of_relax_opts* o);

/* sys: the starting geometry (host).  u, phi: device double* as in of_scf_ground_state (u in:
 * initial guess, out: the ground state at the final positions).  R_out (host, 3 n_atoms):
 * final positions; F_out (host, 3 n_atoms, may be NULL): final forces.  OF_ENOCONV when
 * max_steps is reached first (R_out, F_out and res still describe the last geometry), or when a
 * ground state does not converge. */
of_status of_relax(of_grid* g, const of_system* sys, const of_functional* fn,
                   const of_scf_opts* scf_opts, const of_relax_opts* opts, double* u, double* phi,
                   double* R_out, double* F_out, of_relax_result* res);

/* Vacancy formation energy (Sec. 5.6):
 *   E_vf = E(M-1, 1, (M-1)/M Omega) - ((M-1)/M) E(M, 0, Omega),
 * E(M, n, Omega) the energy of a periodic cell of volume Omega with M occupied sites and n
 * vacancies.  The vacancy cell keeps the volume per atom: its sides and the remaining ion
 * positions are the perfect cell's scaled by ((M-1)/M)^(1/3) about the origin. */
typedef struct {
    double e_perfect;       /* E(M, 0, Omega), Ha */
    double e_unrelaxed;     /* E(M-1, 1, (M-1)/M Omega) at the scaled sites, Ha */
    double e_relaxed;       /* the same after relaxing the vacancy cell's ions (= e_unrelaxed
                               without relaxation), Ha */
    double evf_unrelaxed;   /* e_unrelaxed - (M-1)/M e_perfect, Ha */
    double evf_relaxed;     /* e_relaxed - (M-1)/M e_perfect, Ha */
    double max_force;       /* max_J |F_J| of the vacancy cell at its final positions */
    int relax_steps;        /* NLCG steps of the relaxation (0 without) */
    int evaluations;        /* ground states of the vacancy cell */
} of_vacancy_result;

/* perfect: handle of the perfect cell (sides L); vacancy: a distinct handle with the same grid
 * points, order, stream and device and sides ((M-1)/M)^(1/3) L (to 1e-12 relative; OF_EINVAL
 * otherwise).  sys: the perfect cell's ions (host); site: the index of the ion removed.
 * relax_opts: NULL for the unrelaxed energy only, else the vacancy cell's ions are relaxed at
 * fixed volume as in of_relax.  u_perfect, phi_perfect, u_vacancy, phi_vacancy: device double*
 * fields of the two grids as in of_scf_ground_state (u in: guess, out: ground state).  R_out
 * (host, 3 (M-1), may be NULL): the vacancy cell's final positions.  The two cells' ground
 * states run at once on internal streams; the call synchronises the shared stream.  OF_ENOCONV
 * when a ground state or the relaxation does not converge (res still written). */
of_status of_vacancy_formation(of_grid* perfect, of_grid* vacancy, const of_system* sys, int site,
                               const of_functional* fn, const of_scf_opts* scf_opts,
                               const of_relax_opts* relax_opts, double* u_perfect,
                               double* phi_perfect, double* u_vacancy, double* phi_vacancy,
                               double* R_out, of_vacancy_result* res);

/* Ground states of ncells independent cells at once (same functional and options): grids[c]
 * (distinct handles, one shared stream), systems[c], u[c], phi[c] as in of_scf_ground_state,
 * one result per cell in results[c].  The cells run on up to 8 internal streams driven by host
 * threads, so that their kernels overlap; the call orders them after the work queued on the
 * shared stream and the shared stream after them, and synchronises it.  Returns the first
 * failing cell's status (OF_ENOCONV for a cell that did not converge, results still written). */
of_status of_scf_ground_state_batched(int ncells, of_grid* const* grids, const of_system* systems,
                                      const of_functional* fn, const of_scf_opts* opts,
                                      double* const* u, double* const* phi, of_scf_result* results);

/* Hellmann-Feynman forces of Eq. Force:Nuclei with the overlap correction f^c of App. B:
 * F[3*J + c] (host) for ion J, component c.  phi: device, the ground-state potential.
 * u is accepted for the interface of the paper's statement and not read. */
of_status of_forces(of_grid* g, const of_system* sys, const double* u, const double* phi,
                    double* F);

/* ---- learned preconditioner (Sec. 5.5 asks for better preconditioning; the network is this
 * library's answer, not the paper's) ----
 * A three-layer periodic 3D convolutional network, 1 -> 16 -> 16 -> 1 channels, 3x3x3
 * kernels, exact GELU after the first two layers: y(x) = b + sum_c sum_t W[o][c][t] a[c](x+t),
 * t over (dz, dy, dx) in {-1,0,1}^3 with dz outermost and dx innermost.  Parameters are one
 * float array of of_precond_num_params() = 7809 values: W1[16][27], b1[16], W2[16][16][27],
 * b2[16], W3[16][27], b3.  Kernels keep weights and activations in BF16 and sum in FP32.
 * Applied to a residual r as z = s net(r / s), s = RMS of r.  Trained on residuals r with the
 * loss 1/2 y^T A y - y^T r, y = net(r / s), which equals half the A-norm error of y against
 * A^{-1} r up to a constant, for A = -L_h + c: c = 0 (the default) for the Poisson operator, or
 * c = kf2 |Q| > 0 for a network meant for the shifted kernel system of shift Q (Sec. 3.1; the
 * real positive operator its multigrid preconditioner also inverts).  The handle lives on the
 * current device; every call that takes a grid requires the grid on that device and enqueues
 * on the grid's stream. */
int of_precond_num_params(void);
/* Copies params (host, 7809 floats) to a new handle.  OF_EINVAL on a wrong count. */
of_status of_precond_create(const float* params, int nparams, of_precond** out);
of_status of_precond_destroy(of_precond* P);
/* The operator shift c >= 0 of the training loss (above).  OF_EINVAL for c < 0 or not finite. */
of_status of_precond_set_shift(of_precond* P, double shift);
/* Failure detection: the tensor-core kernels give up waiting for an MMA completion after
 * `seconds` (default 2; 0 <= seconds <= 60), then let the MMAs in flight finish (waiting up to
 * the default limit), free their tensor memory and return; the call that launched them returns
 * OF_ETIMEOUT and the grid and the handle stay usable.  0 makes every such wait give up at
 * once, which exercises that path without a fault. */
of_status of_precond_set_wait_limit(of_precond* P, double seconds);
/* Current FP32 master parameters to host params[7809]. */
of_status of_precond_get_params(of_precond* P, float* params, int nparams);
/* z = s net(r / s) for device float fields r, z (r != z).  Synchronises. */
of_status of_precond_apply(of_grid* g, of_precond* P, const float* r, float* z);
/* Loss of one device float residual r and its parameter gradient (host grad[7809], may be
 * NULL).  Synchronises. */
of_status of_precond_loss_grad(of_grid* g, of_precond* P, const float* r, double* loss, float* grad);
/* Adam (beta 0.9, 0.999) for `steps` steps on mini-batches of `batch` residuals: step s uses
 * samples[order[s * batch + k] * n], k < batch (samples: device, nsamples x n floats; order:
 * host, steps * batch indices in [0, nsamples)).  loss_out: the last mini-batch's mean loss
 * per point.  Synchronises. */
of_status of_precond_train(of_grid* g, of_precond* P, const float* samples, int nsamples,
                           const int* order, int steps, int batch, float lr, double* loss_out);
/* Training data from the solver itself: runs FP32 CG on (-L_h + shift) x = b, b = the device
 * field rho scaled to unit RMS -- for shift = 0 the grid's Poisson system, b = 4 pi (rho -
 * mean rho) -- and copies every stride-th residual, the first one included, to samples[k * n]
 * (device, room for max_samples fields); stops at relative residual 1e-6 or once max_samples
 * are taken; *count = residuals written.  OF_EINVAL for shift < 0.  Synchronises. */
of_status of_precond_collect(of_grid* g, const double* rho, double shift, int stride,
                             int max_samples, float* samples, int* count);

/* Message of the last failure on this host thread ("" if none). */
const char* of_last_error(void);

/* ---- measurement hooks (no counterpart in the paper) ----
 * of_launch_count: kernel launches made by this library so far in the process.
 * of_resource_count: device buffers, pinned host buffers, streams, events and executable CUDA
 * graphs this library has created so far in the process (a call that creates none leaves it
 * unchanged).
 * of_profile_enable: time every sample_every-th launch of each kernel class on the grid's
 * stream with CUDA events (0 stops timing, counting continues); resets the statistics.
 * of_profile_read: synchronises the stream, fills up to max records (one per kernel class
 * seen) and returns their number, -1 on error.  bytes_per_launch is the algorithmic traffic
 * of one launch (fields read plus written, no halo re-reads), averaged over the timed
 * launches: a graph launch of a whole preconditioned pass (classes "mg_pcg_pass_graph",
 * "mg_cocg_pass_graph") counts the iterations it ran. */
typedef struct {
    int kernel_class;
    long long launches;
    long long timed;
    double total_ms;
    double mean_ms;
    double bytes_per_launch;
} of_kernel_stat;

unsigned long long of_launch_count(void);
unsigned long long of_resource_count(void);

/* of_alu_peak: the measured arithmetic rate of this GPU's CUDA cores, the roofline denominator
 * of kernels bound by arithmetic rather than memory (the FP64 Laplacian sweeps).  kind:
 * OF_PEAK_F64 (DFMA), OF_PEAK_F32 (FFMA) or OF_PEAK_F32X2 (packed FP32x2 FMA, two lanes per
 * instruction).  Launches a kernel of 8 independent FMA chains per thread on 8 blocks of 256
 * threads per SM on the given stream (cudaStream_t or NULL) six times (one warm-up, a few ms
 * each) and returns the best rate in *flop_per_s (2 flops per FMA lane).  Creates and
 * destroys two events; synchronises the stream.  OF_EINVAL for an unknown kind. */
enum { OF_PEAK_F64 = 0, OF_PEAK_F32 = 1, OF_PEAK_F32X2 = 2 };
of_status of_alu_peak(int kind, void* stream, double* flop_per_s);
const char* of_kernel_class_name(int kernel_class);
of_status of_profile_enable(of_grid* g, int sample_every);
int of_profile_read(of_grid* g, of_kernel_stat* out, int max);

#ifdef __cplusplus
}
#endif
#endif /* OF_H */
