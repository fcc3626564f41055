// Electronic ground state (Sec. 3.3.1): the constrained non-linear CG of App. C for the inner
// minimisation at fixed V_LR, the kernel map V[u] of Eq. MVF via the shifted solves of Sec. 3.1,
// Anderson mixing of App. D on the fixed point V_LR = V[U(V_LR)], and the ground-state energy
// of Eq. GroundStateEnergy.
//
// Discrete choices shared with the paper's statement:
//  * inner products <a, b> = dV sum a b; the constraint dV sum u^2 = N_e;
//  * vW energy -(lambda/2) <u, L_h u>, so that dE/du = 2 dV H u exactly on the grid;
//  * the NLCG moves along the conjugate direction d_q, restarts every N_restart steps and when
//    the Polak-Ribiere xi <= 0 or d is not a descent direction;
//  * the line energy E(s) of u(s) = sqrt(N_e) (u + s d)/||u + s d|| is exact: by linearity
//    of the Poisson problem phi(s) = c^2 (phi_uu + 2 s phi_ud + s^2 phi_dd) + phi_b, so the
//    Hartree, vW and V_LR parts are polynomials in s times powers of c^2 built from one
//    fused multi-dot pass; only the TF + xc part needs a grid pass per trial s;
//  * Brent's method (own implementation) on a bracket grown from the previous step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "of_functional.cuh"
#include "of_pool.cuh"
#include "of_stencil.cuh"

namespace of {

// indices into g->s.scalars for reduction outputs of this unit
enum {
    SC_UHU = 0, SC_ULU = 1,
    SC_RR = 2, SC_RRP = 3,
    SC_RD = 4, SC_UD = 5, SC_DD = 6, SC_UU = 7,
    SC_DLD = 8, SC_ULD = 9,
    SC_MD = 10,        // 13 line-search moments
    SC_LINE = 25,
    SC_SLOPE = 96,     // 3 sums of the slope line search
    SC_GRADSQ = 100,   // sum of |grad_h u|^2
    SC_EN = 26,        // 4 energy sums
    SC_TLR = 30,
    SC_FP = 32,        // |f|^2, |Vhat|^2
    SC_GRAM = 40,      // Anderson Gram entries
    SC_ZR = 104,       // <z, r>, <z, r_prev> of the preconditioned NLCG
    SC_ZERO = 106      // always 0: the V-cycle's stop flag in the preconditioned NLCG
};

static inline int vb(long long n) { return red_blocks(n, 256 * 4); }

#define GRID_LOOP(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
         i += (long long)gridDim.x * blockDim.x)

struct FnParams {
    double lam, mu, alpha, beta;
};

// ---------------------------------------------------------------- Hamiltonian (stencil op)
// Hu = -(lam/2) L u + (V_TF + V_xc + phi + mu V) u ; Lu = L u ; sums <u,Hu>, <u,Lu>
struct OpHamiltonian {
    const double* u;
    const double* phi;
    const double* V;   // may be null
    double* Hu;
    double* Lu;        // may be null
    FnParams fn;
    RedCtx rc;
    double acc[2];
    __device__ bool begin() { acc[0] = acc[1] = 0.0; return true; }
    __device__ double load(long long i) const { return __ldg(u + i); }
    __device__ void store(long long i, double c, double lap) {
        const double rho = c * c;
        double etf, vtf, exc, vxc;
        thomas_fermi(rho, etf, vtf);
        lda_xc(rho, exc, vxc);
        double pot = vtf + vxc + phi[i];
        if (V) pot += fn.mu * V[i];
        const double h = -0.5 * fn.lam * lap + pot * c;
        Hu[i] = h;
        if (Lu) Lu[i] = lap;
        acc[0] += c * h;
        acc[1] += c * lap;
    }
    __device__ void end() { grid_reduce<2>(acc, rc.partials, rc.counter, rc.out); }
};

// Ld = L d ; sums <d, Ld>, <u, Ld>
struct OpLapDot {
    const double* d;
    const double* u;
    double* Ld;
    RedCtx rc;
    double acc[2];
    __device__ bool begin() { acc[0] = acc[1] = 0.0; return true; }
    __device__ double load(long long i) const { return __ldg(d + i); }
    __device__ void store(long long i, double c, double lap) {
        Ld[i] = lap;
        acc[0] += c * lap;
        acc[1] += u[i] * lap;
    }
    __device__ void end() { grid_reduce<2>(acc, rc.partials, rc.counter, rc.out); }
};

// y = scale * L x (no reduction)
struct OpScaledLap {
    const double* x;
    double* y;
    double scale;
    __device__ bool begin() { return true; }
    __device__ double load(long long i) const { return __ldg(x + i); }
    __device__ void store(long long i, double, double lap) { y[i] = scale * lap; }
    __device__ void end() {}
};

// Energy sums at u: [C_F rho^{5/3}, u L u, eps_xc rho, (rho + b) phi]
struct OpEnergy {
    const double* u;
    const double* b;
    const double* phi;
    RedCtx rc;
    double acc[4];
    __device__ bool begin() { acc[0] = acc[1] = acc[2] = acc[3] = 0.0; return true; }
    __device__ double load(long long i) const { return __ldg(u + i); }
    __device__ void store(long long i, double c, double lap) {
        const double rho = c * c;
        double etf, vtf, exc, vxc;
        thomas_fermi(rho, etf, vtf);
        lda_xc(rho, exc, vxc);
        acc[0] += etf;
        acc[1] += c * lap;
        acc[2] += exc;
        acc[3] += (rho + b[i]) * phi[i];
    }
    __device__ void end() { grid_reduce<4>(acc, rc.partials, rc.counter, rc.out); }
};

// ---------------------------------------------------------------- elementwise kernels
// r = -2 (Hu - eta u) ; sums |r|^2, <r, r_prev>
__global__ void __launch_bounds__(256) k_gradient(long long n, const double* Hu, const double* u,
                                                  const double* eta_raw, double inv_ne_dv,
                                                  const double* rprev, double* r, RedCtx rc) {
    const double eta = (*eta_raw) * inv_ne_dv;
    double acc[2] = {0.0, 0.0};
    GRID_LOOP(i, n) {
        const double v = -2.0 * (Hu[i] - eta * u[i]);
        r[i] = v;
        acc[0] += v * v;
        if (rprev) acc[1] += v * rprev[i];
    }
    grid_reduce<2>(acc, rc.partials, rc.counter, rc.out);
}

// d = r + xi d_prev ; sums <r,d>, <u,d>, <d,d>, <u,u>
__global__ void __launch_bounds__(256) k_direction(long long n, const double* r, const double* dprev,
                                                   double xi, const double* u, double* d, RedCtx rc) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    GRID_LOOP(i, n) {
        const double v = (xi != 0.0 && dprev) ? r[i] + xi * dprev[i] : r[i];
        d[i] = v;
        acc[0] += r[i] * v;
        acc[1] += u[i] * v;
        acc[2] += v * v;
        acc[3] += u[i] * u[i];
    }
    grid_reduce<4>(acc, rc.partials, rc.counter, rc.out);
}

// ---- preconditioned NLCG (nlcg_precond_shift > 0)
// r32 = r / s with s = RMS of r (from the reduced |r|^2), so that the FP32 V-cycle sees unit scale
__global__ void __launch_bounds__(256) k_grad_demote(long long n, const double* r, const double* rr,
                                                     float* r32) {
    const double inv = rsqrt(fmax(*rr / (double)n, 1e-300));
    GRID_LOOP(i, n) r32[i] = (float)(r[i] * inv);
}
// z = s z32 (the preconditioned gradient); sums <z, r>, <z, r_prev>
__global__ void __launch_bounds__(256) k_grad_promote(long long n, const float* z32, const double* rr,
                                                      const double* r, const double* rprev, double* z,
                                                      RedCtx rc) {
    const double s = sqrt(fmax(*rr / (double)n, 1e-300));
    double acc[2] = {0.0, 0.0};
    GRID_LOOP(i, n) {
        const double v = s * (double)z32[i];
        z[i] = v;
        acc[0] += v * r[i];
        if (rprev) acc[1] += v * rprev[i];
    }
    grid_reduce<2>(acc, rc.partials, rc.counter, rc.out);
}
// d = z + xi d_prev ; sums <r,d> (the descent test and dE/ds at s = 0), <u,d>, <d,d>, <u,u>
__global__ void __launch_bounds__(256) k_direction_z(long long n, const double* z, const double* r,
                                                     const double* dprev, double xi, const double* u,
                                                     double* d, RedCtx rc) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    GRID_LOOP(i, n) {
        const double v = (xi != 0.0 && dprev) ? z[i] + xi * dprev[i] : z[i];
        d[i] = v;
        acc[0] += r[i] * v;
        acc[1] += u[i] * v;
        acc[2] += v * v;
        acc[3] += u[i] * u[i];
    }
    grid_reduce<4>(acc, rc.partials, rc.counter, rc.out);
}

// Line-search moments (all raw sums): with A = phi - D, q0 = u^2, q1 = u d, q2 = d^2:
// [q0.A, q0.B, q0.C, q1.B, q1.C, q2.C, q0.D, q1.D, q2.D, V.q0, V.q1, V.q2, b.D]
__global__ void __launch_bounds__(256) k_line_moments(long long n, const double* u, const double* d,
                                                      const double* V, const double* phi,
                                                      const double* D, const double* B,
                                                      const double* C, const double* b, RedCtx rc) {
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    GRID_LOOP(i, n) {
        const double uu = u[i], dd = d[i];
        const double q0 = uu * uu, q1 = uu * dd, q2 = dd * dd;
        const double Di = D[i], Ai = phi[i] - Di, Bi = B[i], Ci = C[i];
        acc[0] += q0 * Ai;
        acc[1] += q0 * Bi;
        acc[2] += q0 * Ci;
        acc[3] += q1 * Bi;
        acc[4] += q1 * Ci;
        acc[5] += q2 * Ci;
        acc[6] += q0 * Di;
        acc[7] += q1 * Di;
        acc[8] += q2 * Di;
        if (V) {
            const double v = V[i];
            acc[9] += v * q0;
            acc[10] += v * q1;
            acc[11] += v * q2;
        }
        acc[12] += b[i] * Di;
    }
    grid_reduce<13>(acc, rc.partials, rc.counter, rc.out);
}

// sum of TF + xc energy densities at rho = c2 (u + s d)^2
__global__ void __launch_bounds__(256) k_line_energy(long long n, const double* u, const double* d,
                                                     double s, double c2, RedCtx rc) {
    double acc[1] = {0.0};
    GRID_LOOP(i, n) {
        const double w = u[i] + s * d[i];
        acc[0] += tf_xc_energy(c2 * w * w);
    }
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

// With w = u + s d and rho = c2 w^2: sums of e(rho), v(rho) w^2 and v(rho) w d, e the TF + xc
// energy density and v = de/drho.  The line derivative of the TF + xc energy follows from them.
__global__ void __launch_bounds__(256) k_line_energy_slope(long long n, const double* u,
                                                           const double* d, double s, double c2,
                                                           RedCtx rc) {
    double acc[3] = {0.0, 0.0, 0.0};
    GRID_LOOP(i, n) {
        const double di = d[i];
        const double w = fma(s, di, u[i]);
        double e, v;
        tf_xc_energy_slope(c2 * w * w, e, v);
        const double vw = v * w;
        acc[0] += e;
        acc[1] += vw * w;
        acc[2] += vw * di;
    }
    grid_reduce<3>(acc, rc.partials, rc.counter, rc.out);
}

// u <- c (u + s d) ; phi <- c^2 (phi - D + 2 s B + s^2 C) + D
__global__ void k_step(long long n, double* u, const double* d, double* phi, const double* D,
                       const double* B, const double* C, double s, double c) {
    const double c2 = c * c;
    GRID_LOOP(i, n) {
        u[i] = c * (u[i] + s * d[i]);
        const double Di = D[i];
        phi[i] = c2 * (phi[i] - Di + 2.0 * s * B[i] + s * s * C[i]) + Di;
    }
}

// Starting points of the next line's Poisson solves from the last ones: with u = c (u_p + s d_p)
// and d = z + xi d_p, linearity gives phi(u d) = xi c (phi(u_p d_p) + s phi(d_p^2)) + phi(u z) and
// phi(d^2) = xi^2 phi(d_p^2) + (terms in z); the known parts start the solves.
__global__ void k_line_guess(long long n, double* B, double* C, double a1, double s, double a2) {
    GRID_LOOP(i, n) {
        const double Ci = C[i];
        B[i] = a1 * (B[i] + s * Ci);
        C[i] = a2 * Ci;
    }
}

__global__ void k_scale(long long n, double* x, double a) {
    GRID_LOOP(i, n) x[i] *= a;
}

// y = u^2 + b
__global__ void k_density_plus(long long n, const double* u, const double* b, double* y) {
    GRID_LOOP(i, n) y[i] = u[i] * u[i] + b[i];
}

// g_a = max(u, floor)^{2 alpha}, g_b = max(u, floor)^{2 beta}
__global__ void k_powers(long long n, const double* u, double two_a, double two_b, double* ga,
                         double* gb) {
    GRID_LOOP(i, n) {
        const double uf = fmax(u[i], OF_U_FLOOR);
        ga[i] = pow(uf, two_a);
        gb[i] = pow(uf, two_b);
    }
}

// The density powers of the second-order kernel term: g[j] = u^{2(j + alpha)} and
// g[3 + j] = u^{2(j + beta)}, j = 0..2 (u raised to the floor)
__global__ void k_powers6(long long n, const double* u, double two_a, double two_b, double* g) {
    GRID_LOOP(i, n) {
        const double uf = fmax(u[i], OF_U_FLOOR);
        const double rho = uf * uf;
        const double a = pow(uf, two_a), b = pow(uf, two_b);
        g[i] = a;
        g[n + i] = a * rho;
        g[2 * n + i] = a * rho * rho;
        g[3 * n + i] = b;
        g[4 * n + i] = b * rho;
        g[5 * n + i] = b * rho * rho;
    }
}

// Second-order (L = 2) kernel term, summed over potentials: the potential p is
// V_p = sum over its conjugate pairs of 2 Re W[p][k]; with g the six density powers,
//   V_LR = (C_F / rho) sum_p V_p sum_j cv[p][j] g_j,   sum of sum_p V_p sum_j ct[p][j] g_j,
// cv and ct holding C_mnpq (times m - p + alpha or n - q + beta for cv) of the terms that
// pair potential p with power j.
constexpr int LR_MAX_POT = 16;
struct LrSum {
    int npot, npairs;
    const double2* W[LR_MAX_POT][4];
    double cv[LR_MAX_POT][6];
    double ct[LR_MAX_POT][6];
};
__global__ void __launch_bounds__(256) k_lr_assemble2(long long n, const double* u, const double* g,
                                                      LrSum S, double* vlr, RedCtx rc) {
    double acc[1] = {0.0};
    GRID_LOOP(i, n) {
        double gj[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) gj[j] = g[j * n + i];
        double vl = 0.0, te = 0.0;
#pragma unroll
        for (int p = 0; p < LR_MAX_POT; ++p) {
            if (p < S.npot) {
                double V = 0.0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < S.npairs) V += 2.0 * S.W[p][k][i].x;
                double a = 0.0, b = 0.0;
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    a = fma(S.cv[p][j], gj[j], a);
                    b = fma(S.ct[p][j], gj[j], b);
                }
                vl = fma(a, V, vl);
                te = fma(b, V, te);
            }
        }
        const double uf = fmax(u[i], OF_U_FLOOR);
        vlr[i] = OF_CF * vl / (uf * uf);
        acc[0] += te;
    }
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

// V_LR = C_F [alpha u^{2(alpha-1)} V_beta + beta u^{2(beta-1)} V_alpha], V_e = sum over
// conjugate pairs of 2 Re W ; sum of u^{2 alpha} V_beta + u^{2 beta} V_alpha.
struct PairPtrs {
    const double2* Wa[4];
    const double2* Wb[4];
    int npairs;
};
__global__ void __launch_bounds__(256) k_lr_assemble(long long n, const double* u, PairPtrs W,
                                                     double alpha, double beta, double* vlr,
                                                     RedCtx rc) {
    double acc[1] = {0.0};
    GRID_LOOP(i, n) {
        double Va = 0.0, Vb = 0.0;
        for (int k = 0; k < W.npairs; ++k) {
            Va += 2.0 * W.Wa[k][i].x;
            Vb += 2.0 * W.Wb[k][i].x;
        }
        const double uf = fmax(u[i], OF_U_FLOOR);
        const double ra = pow(uf, 2.0 * alpha), rb = pow(uf, 2.0 * beta);
        vlr[i] = OF_CF * (alpha * (ra / (uf * uf)) * Vb + beta * (rb / (uf * uf)) * Va);
        acc[0] += ra * Vb + rb * Va;
    }
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

// f = Vhat - V ; sums |f|^2, |Vhat|^2
__global__ void __launch_bounds__(256) k_fp_residual(long long n, const double* Vhat, const double* V,
                                                     double* f, RedCtx rc) {
    double acc[2] = {0.0, 0.0};
    GRID_LOOP(i, n) {
        const double v = Vhat[i] - V[i];
        f[i] = v;
        acc[0] += v * v;
        acc[1] += Vhat[i] * Vhat[i];
    }
    grid_reduce<2>(acc, rc.partials, rc.counter, rc.out);
}

// y = a - b
__global__ void k_diff(long long n, const double* a, const double* b, double* y) {
    GRID_LOOP(i, n) y[i] = a[i] - b[i];
}

struct HistPtrs {
    const double* S[8];
    const double* Y[8];
    double g[8];
    int m;
};

// Gram entries Y_a . Y_b (a <= b, row-major upper triangle) then Y_a . f
template <int M>
__global__ void __launch_bounds__(256) k_gram(long long n, HistPtrs H, const double* f, RedCtx rc) {
    constexpr int K = M * (M + 1) / 2 + M;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    GRID_LOOP(i, n) {
        double y[M];
#pragma unroll
        for (int a = 0; a < M; ++a) y[a] = H.Y[a][i];
        int k = 0;
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b) acc[k++] += y[a] * y[b];
        const double fi = f[i];
#pragma unroll
        for (int a = 0; a < M; ++a) acc[k++] += y[a] * fi;
    }
    grid_reduce<K>(acc, rc.partials, rc.counter, rc.out);
}

// V <- V + zeta f - sum_a g_a (S_a + zeta Y_a)
__global__ void k_anderson_update(long long n, double* V, const double* f, double zeta, HistPtrs H) {
    GRID_LOOP(i, n) {
        double v = V[i] + zeta * f[i];
        for (int a = 0; a < H.m; ++a) v -= H.g[a] * (H.S[a][i] + zeta * H.Y[a][i]);
        V[i] = v;
    }
}

// ---------------------------------------------------------------- host helpers
static double sc(of_grid* g, int i) {
    double v;
    fetch_scalars(g, i, 1, &v);
    return v;
}

static FnParams fn_params(const of_functional* fn) {
    return FnParams{fn->lambda, fn->mu, fn->alpha, fn->beta};
}

// Brent's method for a minimum inside the bracket a < b < c with f(b) < f(a), f(c)
// (parabolic interpolation through the three best points, golden-section fallback).
template <class F>
static double brent_minimise(F&& f, double a, double b, double c, double fb, double tol,
                             int max_iter, int& evals) {
    const double cgold = 0.3819660112501051;
    double lo = std::min(a, c), hi = std::max(a, c);
    double x = b, w = b, v = b, fx = fb, fw = fb, fv = fb;
    double e = 0.0, step = 0.0;
    for (int it = 0; it < max_iter; ++it) {
        const double xm = 0.5 * (lo + hi);
        const double tol1 = tol * std::fabs(x) + 1e-11, tol2 = 2.0 * tol1;
        if (std::fabs(x - xm) <= tol2 - 0.5 * (hi - lo)) break;
        bool golden = true;
        if (std::fabs(e) > tol1) {
            double r = (x - w) * (fx - fv);
            double q = (x - v) * (fx - fw);
            double p = (x - v) * q - (x - w) * r;
            q = 2.0 * (q - r);
            if (q > 0.0) p = -p;
            q = std::fabs(q);
            const double etemp = e;
            if (std::fabs(p) < std::fabs(0.5 * q * etemp) && p > q * (lo - x) && p < q * (hi - x)) {
                e = step;
                step = p / q;
                const double u = x + step;
                if (u - lo < tol2 || hi - u < tol2) step = (xm - x >= 0) ? tol1 : -tol1;
                golden = false;
            }
        }
        if (golden) {
            e = (x >= xm) ? lo - x : hi - x;
            step = cgold * e;
        }
        const double u = (std::fabs(step) >= tol1) ? x + step : x + (step >= 0 ? tol1 : -tol1);
        const double fu = f(u);
        ++evals;
        if (fu <= fx) {
            if (u >= x) lo = x; else hi = x;
            v = w; fv = fw;
            w = x; fw = fx;
            x = u; fx = fu;
        } else {
            if (u < x) lo = u; else hi = u;
            if (fu <= fw || w == x) {
                v = w; fv = fw;
                w = u; fw = fu;
            } else if (fu <= fv || v == x || v == w) {
                v = u; fv = fu;
            }
        }
    }
    return x;
}

// Bracket from s = 0 along increasing s (golden expansion while f decreases, shrink while it
// does not), then Brent.  Returns 0 when no decrease is found.
template <class F>
static double line_minimum(F&& f, double s_try, double tol, int& evals) {
    const double gold = 1.618033988749895;
    const double f0 = f(0.0);
    double b = std::fabs(s_try), fb = f(b);
    double a = 0.0, c, fc;
    evals += 2;
    if (fb < f0) {
        c = b * (1.0 + gold);
        fc = f(c);
        ++evals;
        int k = 0;
        while (fc < fb && k < 60) {
            a = b;
            b = c; fb = fc;
            c = b + gold * (b - a);
            fc = f(c);
            ++evals;
            ++k;
        }
        if (fc < fb) return c;
        if (!(fc > fb)) return b;   // flat to rounding between b and c
    } else {
        c = b; fc = fb;
        b = c / (1.0 + gold);
        fb = f(b);
        ++evals;
        int k = 0;
        while (fb >= f0 && k < 60) {
            c = b; fc = fb;
            b = c / (1.0 + gold);
            fb = f(b);
            ++evals;
            ++k;
        }
        if (fb >= f0) return 0.0;
        a = 0.0;
    }
    return brent_minimise(f, a, b, c, fb, tol, 100, evals);
}

// Minimises E along s >= 0 from E' alone (E and E' come from one pass; only the slope is used,
// since near convergence E changes along the line by less than its rounding).  g0 = E'(0) < 0.
// The trial step s_try is extended while E' stays negative (secant extrapolation of E',
// between 1.5x and 8x per extension); inside the bracket the root of E' is found by the secant
// method with the Illinois modification.  Stops when |E'| <= tol |g0| (for E' linear in s, a
// relative error tol in the step) or the bracket is narrower than tol times its right end.
// Returns 0 when no step with E' < 0 beyond s = 0 is found.
template <class F>
static double line_minimum_slope(F&& f, double g0, double s_try, double tol, int& evals) {
    if (!(g0 < 0.0)) return 0.0;
    const double gtol = -tol * g0;
    double a = 0.0, ga = g0;
    double b = std::fabs(s_try) > 0.0 ? std::fabs(s_try) : 1e-2, gb;
    double e;
    f(b, e, gb);
    ++evals;
    for (int k = 0; gb < 0.0; ++k) {   // still descending at b: extend
        if (-gb <= gtol) return b;
        if (k == 60) return b;
        double next = 8.0 * b;
        if (gb > ga) next = std::min(8.0 * b, std::max(1.5 * b, b - gb * (b - a) / (gb - ga)));
        a = b;
        ga = gb;
        b = next;
        f(b, e, gb);
        ++evals;
    }
    if (gb <= gtol) return b;
    // bracket: E'(a) < 0 <= E'(b)
    double Ga = ga, Gb = gb;   // end values of the secant, halved by the Illinois rule
    int kept = 0;              // +1: a was kept by the last step, -1: b was
    for (int it = 0; it < 40; ++it) {
        double m = a - Ga * (b - a) / (Gb - Ga);
        if (!(m > a && m < b)) m = 0.5 * (a + b);
        double gm;
        f(m, e, gm);
        ++evals;
        if (std::fabs(gm) <= gtol) return m;
        if (gm < 0.0) {
            a = m;
            Ga = gm;
            if (kept == -1) Gb *= 0.5;
            kept = -1;
        } else {
            b = m;
            Gb = gm;
            if (kept == 1) Ga *= 0.5;
            kept = 1;
        }
        if (b - a <= tol * b) return 0.5 * (a + b);
        if (a == 0.0 && b <= 1e-9 * std::fabs(s_try)) return 0.0;   // E' > 0 right of 0
    }
    return a;
}

// Device vectors used by the ground-state driver.
struct ScfVecs {
    double *Hu, *Lu, *r, *rp, *d, *dp, *B, *C, *Ld, *b, *D, *rho, *V, *Vhat;
};

static ScfVecs scf_vecs(of_grid* g) {
    const size_t bytes = sizeof(double) * (size_t)g->d.n;
    ScfVecs v;
    double** p[] = {&v.Hu, &v.Lu, &v.r, &v.rp, &v.d, &v.dp, &v.B, &v.C, &v.Ld, &v.b, &v.D,
                    &v.rho, &v.V, &v.Vhat};
    for (int k = 0; k < 14; ++k) *p[k] = (double*)ws(g, WS_S0 + k, bytes);
    return v;
}

struct ScfStats {
    int nlcg = 0, poisson = 0, kernel = 0, line = 0;
    double last_residual = 0.0;
};

// Poisson solve of rho = a*b (or a when b == null) with warm start in phi.
static void poisson_into(of_grid* g, const double* a, const double* b, double* phi,
                         const KrylovOpts& o, ScfStats& st) {
    of_solve_info info{};
    of_status s = b ? poisson_product(g, a, b, phi, o, &info) : poisson(g, a, phi, o, &info);
    st.poisson += info.iterations;
    if (s != OF_OK && s != OF_ENOCONV) throw Error{s};
}

// The twin handle of g (same grid, own workspace, graphs and stream), created on first use,
// with the profiling state of g.
static of_grid* twin_of(of_grid* g) {
    if (!g->twin) {
        of_grid* t = nullptr;
        OF_CUDA(cudaStreamCreateWithFlags(&g->twin_stream, cudaStreamNonBlocking));
        OF_CUDA(cudaEventCreateWithFlags(&g->twin_in, cudaEventDisableTiming));
        OF_CUDA(cudaEventCreateWithFlags(&g->twin_out, cudaEventDisableTiming));
        for (int k = 0; k < 3; ++k) note_resource();
        const of_status s = of_grid_create(g->d.n1, g->d.n2, g->d.n3, g->L[0], g->L[1], g->L[2], g->N,
                                           g->twin_stream, &t);
        if (s != OF_OK) throw Error{s};
        g->twin = t;
        if (g->prof && g->prof->every > 0) of_profile_enable(t, g->prof->every);
    }
    g->twin->stream = g->twin_stream;
    return g->twin;
}

// The host thread that runs the second half of every pair on a handle: started with the
// handle's first pair, idle on a condition variable between pairs, joined when the handle is
// destroyed (a thread per pair cost a thread start every NLCG step and kernel map).
struct PairWorker {
    std::thread th;
    std::mutex m;
    std::condition_variable cv;
    std::function<void()> task;
    bool has_task = false, busy = false, stop = false;
    explicit PairWorker(int device) {
        th = std::thread([this, device]() {
            cudaSetDevice(device);
            for (;;) {
                std::function<void()> f;
                {
                    std::unique_lock<std::mutex> lk(m);
                    cv.wait(lk, [this] { return has_task || stop; });
                    if (!has_task) return;
                    f = std::move(task);
                    has_task = false;
                }
                f();   // never throws: the tasks of run_pair catch everything
                {
                    std::lock_guard<std::mutex> lk(m);
                    busy = false;
                }
                cv.notify_all();
            }
        });
    }
    void post(std::function<void()> f) {
        {
            std::lock_guard<std::mutex> lk(m);
            task = std::move(f);
            has_task = true;
            busy = true;
        }
        cv.notify_all();
    }
    void wait() {
        std::unique_lock<std::mutex> lk(m);
        cv.wait(lk, [this] { return !busy; });
    }
    ~PairWorker() {
        {
            std::lock_guard<std::mutex> lk(m);
            stop = true;
        }
        cv.notify_all();
        th.join();
    }
};

static void destroy_pair_worker(void* p) { delete static_cast<PairWorker*>(p); }

static PairWorker* pair_worker(of_grid* g) {
    if (!g->worker) {
        g->worker = new PairWorker(g->device);
        g->worker_destroy = destroy_pair_worker;
    }
    return static_cast<PairWorker*>(g->worker);
}

// Two independent pieces of work at once: first(g) on g's stream in this thread, second(t) on
// the twin handle t (its own stream and workspace) in the handle's worker thread.  Both are
// latency-bound solves at the benchmark's sizes, so they overlap on the GPU.  The twin's
// stream starts after the work queued on g's stream, which waits for the twin before it goes
// on.  An error of either side is rethrown after both have finished.
template <class First, class Second>
static void run_pair(of_grid* g, First&& first, Second&& second) {
    of_grid* t = twin_of(g);
    PairWorker* w = pair_worker(g);
    OF_CUDA(cudaEventRecord(g->twin_in, g->stream));
    OF_CUDA(cudaStreamWaitEvent(t->stream, g->twin_in, 0));
    of_status err2 = OF_OK;
    std::string msg2;
    w->post([&]() {
        try {
            second(t);
        } catch (const Error& e) {
            err2 = e.code;
            msg2 = of_last_error();
        } catch (...) {
            err2 = OF_ECUDA;
            msg2 = "unexpected exception in the second solve of a pair";
        }
    });
    of_status err1 = OF_OK;
    try {
        first(g);
    } catch (const Error& e) {
        err1 = e.code;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in a paired solve");
        err1 = OF_ENOMEM;
    } catch (...) {   // whatever it was, the worker finishes before anything leaves
        set_error("unexpected exception in a paired solve");
        err1 = OF_ECUDA;
    }
    w->wait();
    OF_CUDA(cudaEventRecord(g->twin_out, t->stream));
    OF_CUDA(cudaStreamWaitEvent(g->stream, g->twin_out, 0));
    if (err1 != OF_OK) throw Error{err1};
    if (err2 != OF_OK) {
        set_error("%s", msg2.c_str());
        throw Error{err2};
    }
}

// Up to GROUP_MAX independent solves at once: task 0 on g in this thread, task i on the i-th
// handle of g's twin chain (g->twin, its twin, ...) in the worker thread of the handle before
// it.  The chain's streams start after the work queued on g's stream, which waits for all of
// them before it goes on.  The first error is rethrown after every task has finished.
constexpr int GROUP_MAX = 4;

static void run_group(of_grid* g, int ntasks, const std::function<void(of_grid*, int)>& task) {
    OF_REQUIRE(ntasks >= 1 && ntasks <= GROUP_MAX, OF_EINVAL, "run_group: %d tasks", ntasks);
    of_grid* H[GROUP_MAX] = {g};
    for (int i = 1; i < ntasks; ++i) H[i] = twin_of(H[i - 1]);
    if (ntasks > 1) {
        OF_CUDA(cudaEventRecord(g->twin_in, g->stream));
        for (int i = 1; i < ntasks; ++i) OF_CUDA(cudaStreamWaitEvent(H[i]->stream, g->twin_in, 0));
    }
    of_status err[GROUP_MAX] = {};
    std::string msg[GROUP_MAX];
    PairWorker* w[GROUP_MAX] = {};
    for (int i = 1; i < ntasks; ++i) {
        w[i] = pair_worker(H[i - 1]);
        w[i]->post([&, i]() {
            try {
                task(H[i], i);
            } catch (const Error& e) {
                err[i] = e.code;
                msg[i] = of_last_error();
            } catch (...) {
                err[i] = OF_ECUDA;
                msg[i] = "unexpected exception in a grouped solve";
            }
        });
    }
    try {
        task(g, 0);
    } catch (const Error& e) {
        err[0] = e.code;
        msg[0] = of_last_error();
    } catch (const std::bad_alloc&) {
        err[0] = OF_ENOMEM;
        msg[0] = "host allocation failed in a grouped solve";
    } catch (...) {   // whatever it was, the workers finish before anything leaves
        err[0] = OF_ECUDA;
        msg[0] = "unexpected exception in a grouped solve";
    }
    for (int i = 1; i < ntasks; ++i) w[i]->wait();
    for (int i = 1; i < ntasks; ++i) {
        OF_CUDA(cudaEventRecord(H[i - 1]->twin_out, H[i]->stream));
        OF_CUDA(cudaStreamWaitEvent(g->stream, H[i - 1]->twin_out, 0));
    }
    for (int i = 0; i < ntasks; ++i)
        if (err[i] != OF_OK) {
            set_error("%s", msg[i].c_str());
            throw Error{err[i]};
        }
}

// The two line-energy Poisson solves of products, phi1 for rho = a1 b1 and phi2 for
// rho = a2 b2, at once (run_pair); pre(g) is queued on g's stream ahead of the first solve, so
// that it overlaps the second.
template <class Pre>
static void poisson_pair(of_grid* g, const double* a1, const double* b1, double* phi1,
                         const double* a2, const double* b2, double* phi2, const KrylovOpts& o,
                         ScfStats& st, Pre&& pre) {
    if (o.precond) {   // a learned preconditioner's buffers serve one solve at a time; its
                       // flexible CG reduces into more scalar slots, so pre goes last
        poisson_into(g, a1, b1, phi1, o, st);
        poisson_into(g, a2, b2, phi2, o, st);
        pre(g);
        return;
    }
    ScfStats st2;
    run_pair(g,
             [&](of_grid* h) {
                 pre(h);
                 poisson_into(h, a1, b1, phi1, o, st);
             },
             [&](of_grid* h) { poisson_into(h, a2, b2, phi2, o, st2); });
    st.poisson += st2.poisson;
}

// y = -L_h x + s x (FP32), the numerator of the two-shift NLCG preconditioner
struct OpShiftedNegLap32 {
    const float* x;
    float* y;
    float s;
    __device__ bool begin() { return true; }
    __device__ float load(long long i) const { return x[i]; }
    __device__ void store(long long i, float c, float lap) { y[i] = fmaf(s, c, -lap); }
    __device__ void end() {}
};

// Tolerance of the Poisson re-solve after an NLCG step, relative to the normalised gradient
// norm (tuned on the 108-atom cell)
constexpr double RESOLVE_FACTOR = 1e-3;

// Inner minimisation U(V) (App. C).  u, phi in/out.  Returns true when converged.
static bool nlcg(of_grid* g, const FnParams& fn, double Ne, ScfVecs& v, double* u, double* phi,
                 const double* V, double tol, int max_iter, int n_restart, double line_tol,
                 int line_search, const KrylovOpts& po, ScfStats& st, double pshift, double plow) {
    const long long n = g->d.n;
    const double dV = g->dV;
    // preconditioned NLCG: buffers of the gradient in FP32, its V-cycle and the FP64 direction
    struct {
        float *r32 = nullptr, *z32 = nullptr;
        double* z = nullptr;
    } pc;
    double zr_prev = 0.0;
    if (pshift > 0.0 && mg_available(g)) {
        char* p = (char*)ws(g, WS_NLCGP, (sizeof(float) * 2 + sizeof(double)) * (size_t)n + 256);
        pc.z = (double*)p;
        pc.r32 = (float*)(p + sizeof(double) * (size_t)n);
        pc.z32 = pc.r32 + n;
    } else {
        pshift = 0.0;
    }
    const int nb = vb(n);
    // normalise u and solve for its potential
    launch(k_sum_product, nb, 256, g->stream, n, u, u, red_ctx(g, SC_UU));
    OF_LAUNCH_CHECK();
    const double uu0 = sc(g, SC_UU) * dV;
    OF_REQUIRE(uu0 > 0 && std::isfinite(uu0), OF_EINVAL, "initial u has zero or non-finite norm");
    launch(k_scale, nb, 256, g->stream, n, u, std::sqrt(Ne / uu0));
    launch(k_density_plus, nb, 256, g->stream, n, u, v.b, v.rho);
    OF_LAUNCH_CHECK();
    poisson_into(g, v.rho, nullptr, phi, po, st);

    double rr_prev = 0.0, s_prev = 1e-2, c_prev = 0.0;
    bool converged = false;
    for (int q = 0; q <= max_iter; ++q) {
        launch_stencil<double, 2>(g, g->w64,
                                  OpHamiltonian{u, phi, fn.mu != 0.0 ? V : nullptr, v.Hu, v.Lu, fn,
                                                red_ctx(g, SC_UHU)});
        launch(k_gradient, nb, 256, g->stream, n, v.Hu, u, g->s.scalars + SC_UHU, dV / Ne,
                                              q > 0 ? v.rp : nullptr, v.r, red_ctx(g, SC_RR));
        OF_LAUNCH_CHECK();
        double h[4];
        fetch_scalars(g, SC_UHU, 4, h);
        const double rr = h[2], rrp = h[3];
        st.last_residual = std::sqrt(dV * rr / Ne);
        if (st.last_residual < tol) { converged = true; break; }
        if (q == max_iter) break;
        double xi = 0.0;
        double m[4];
        if (pshift > 0.0) {
            // preconditioned direction: z = M^{-1} r with M^{-1} one V-cycle of -L_h + pshift,
            // or (-L_h + plow) times two of them (FP32 on the gradient scaled to unit RMS),
            // Polak-Ribiere in the preconditioned form xi = <z, r - r_prev> / <z_prev, r_prev>,
            // d = z + xi d_prev
            launch(k_grad_demote, nb, 256, g->stream, n, (const double*)v.r,
                   (const double*)(g->s.scalars + SC_RR), pc.r32);
            mg_vcycle_real_shifted(g, pc.r32, pc.z32, g->s.scalars + SC_ZERO, pshift);
            if (plow > 0.0) {
                mg_vcycle_real_shifted(g, pc.z32, pc.r32, g->s.scalars + SC_ZERO, pshift);
                launch_stencil<float, 2>(g, g->w32, OpShiftedNegLap32{pc.r32, pc.z32, (float)plow});
            }
            launch(k_grad_promote, nb, 256, g->stream, n, (const float*)pc.z32,
                   (const double*)(g->s.scalars + SC_RR), (const double*)v.r,
                   q > 0 ? (const double*)v.rp : nullptr, pc.z, red_ctx(g, SC_ZR));
            OF_LAUNCH_CHECK();
            double zr[2];
            fetch_scalars(g, SC_ZR, 2, zr);
            if (q > 0 && q % n_restart != 0 && zr_prev > 0.0) {
                xi = (zr[0] - zr[1]) / zr_prev;
                if (!(xi > 0.0)) xi = 0.0;
            }
            zr_prev = zr[0];
            launch(k_direction_z, nb, 256, g->stream, n, (const double*)pc.z, (const double*)v.r,
                   (const double*)v.dp, xi, u, v.d, red_ctx(g, SC_RD));
            OF_LAUNCH_CHECK();
            fetch_scalars(g, SC_RD, 4, m);
        } else {
            if (q > 0 && q % n_restart != 0) {
                xi = (rr - rrp) / rr_prev;
                if (!(xi > 0.0)) xi = 0.0;
            }
            launch(k_direction, nb, 256, g->stream, n, v.r, v.dp, xi, u, v.d, red_ctx(g, SC_RD));
            OF_LAUNCH_CHECK();
            fetch_scalars(g, SC_RD, 4, m);
        }
        if (!(m[0] > 0.0) && (xi != 0.0 || pshift > 0.0)) {   // not a descent direction: restart
            xi = 0.0;                                            // along r
            launch(k_direction, nb, 256, g->stream, n, v.r, v.dp, 0.0, u, v.d, red_ctx(g, SC_RD));
            OF_LAUNCH_CHECK();
            fetch_scalars(g, SC_RD, 4, m);
        }
        // phi_ud and phi_dd only shape the line energy E(s) (the Hartree moments) and the
        // starting point of the re-solve below, which sets phi for the gradient and the energy
        // to the full tolerance.  They are solved to min(1e-5, 1e-2 x the normalised gradient
        // norm), which resolves dE/ds well within the line search's tolerance; if the line
        // search finds no decrease, the step is repeated with both solved to the full tolerance.
        launch(k_line_guess, nb, 256, g->stream, n, v.B, v.C, xi * c_prev, s_prev, xi * xi);
        const double ud = m[1] * dV, dd = m[2] * dV, uu = m[3] * dV;
        double dLd = 0, uLd = 0, uLu_ = 0, M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0;
        double N0 = 0, N1 = 0, N2 = 0, Vq0 = 0, Vq1 = 0, Vq2 = 0, bD = 0;
        auto prepare_line = [&](double tol_line) {
            KrylovOpts pl = po;
            pl.tol = std::max(po.tol, tol_line);
            // L d with d^T L d and u^T L d (slots untouched by the solves) beside the twin's solve
            poisson_pair(g, u, v.d, v.B, v.d, v.d, v.C, pl, st, [&](of_grid* h) {
                launch_stencil<double, 2>(h, h->w64, OpLapDot{v.d, u, v.Ld, red_ctx(h, SC_DLD)});
            });
            launch(k_line_moments, nb, 256, g->stream, n, u, v.d, fn.mu != 0.0 ? V : nullptr, phi,
                   v.D, v.B, v.C, v.b, red_ctx(g, SC_MD));
            OF_LAUNCH_CHECK();
            double mo[17];
            fetch_scalars(g, SC_DLD, 15, mo);   // DLD, ULD, then the 13 moments
            double uLu;
            fetch_scalars(g, SC_ULU, 1, &uLu);
            dLd = mo[0] * dV;
            uLd = mo[1] * dV;
            uLu_ = uLu * dV;
            const double* M = mo + 2;
            M00 = M[0] * dV; M01 = M[1] * dV; M02 = M[2] * dV; M11 = M[3] * dV;
            M12 = M[4] * dV; M22 = M[5] * dV; N0 = M[6] * dV; N1 = M[7] * dV;
            N2 = M[8] * dV; Vq0 = M[9] * dV; Vq1 = M[10] * dV; Vq2 = M[11] * dV;
            bD = M[12] * dV;
        };
        auto energy = [&](double s) -> double {
            const double c2 = Ne / (uu + 2.0 * s * ud + s * s * dd);
            ProfScope ps(g, PC_LINE, 2.0 * sizeof(double) * (double)n);
            launch(k_line_energy, nb, 256, g->stream, n, u, v.d, s, c2, red_ctx(g, SC_LINE));
            OF_LAUNCH_CHECK();
            const double tfxc = sc(g, SC_LINE) * dV;
            const double vw = -0.5 * fn.lam * c2 * (uLu_ + 2.0 * s * uLd + s * s * dLd);
            const double vl = fn.mu != 0.0 ? fn.mu * c2 * (Vq0 + 2.0 * s * Vq1 + s * s * Vq2) : 0.0;
            const double quart = M00 + 4.0 * s * M01 + 2.0 * s * s * M02 + 4.0 * s * s * M11 +
                                 4.0 * s * s * s * M12 + s * s * s * s * M22;
            const double hart = 0.5 * c2 * c2 * quart + c2 * (N0 + 2.0 * s * N1 + s * s * N2) + 0.5 * bD;
            return tfxc + vw + vl + hart;
        };
        // E and dE/ds together (slope line search): the TF + xc sums of k_line_energy_slope
        // and the derivatives of the closed-form vW, kernel and Hartree terms
        auto energy_slope = [&](double s, double& E, double& G) {
            const double q = uu + 2.0 * s * ud + s * s * dd;
            const double c2 = Ne / q;
            const double c2p = -c2 * (2.0 * ud + 2.0 * s * dd) / q;
            ProfScope ps(g, PC_LINE, 2.0 * sizeof(double) * (double)n);
            launch(k_line_energy_slope, nb, 256, g->stream, n, u, v.d, s, c2, red_ctx(g, SC_SLOPE));
            OF_LAUNCH_CHECK();
            double t[3];
            fetch_scalars(g, SC_SLOPE, 3, t);
            const double tfxc = t[0] * dV, tfxc_p = (c2p * t[1] + 2.0 * c2 * t[2]) * dV;
            const double P = uLu_ + 2.0 * s * uLd + s * s * dLd, Pp = 2.0 * uLd + 2.0 * s * dLd;
            const double R = Vq0 + 2.0 * s * Vq1 + s * s * Vq2, Rp = 2.0 * Vq1 + 2.0 * s * Vq2;
            const double quart = M00 + 4.0 * s * M01 + 2.0 * s * s * M02 + 4.0 * s * s * M11 +
                                 4.0 * s * s * s * M12 + s * s * s * s * M22;
            const double quart_p = 4.0 * M01 + 4.0 * s * M02 + 8.0 * s * M11 +
                                   12.0 * s * s * M12 + 4.0 * s * s * s * M22;
            const double Nq = N0 + 2.0 * s * N1 + s * s * N2, Nq_p = 2.0 * N1 + 2.0 * s * N2;
            E = tfxc - 0.5 * fn.lam * c2 * P + fn.mu * c2 * R + 0.5 * c2 * c2 * quart + c2 * Nq + 0.5 * bD;
            G = tfxc_p - 0.5 * fn.lam * (c2p * P + c2 * Pp) + fn.mu * (c2p * R + c2 * Rp) +
                c2 * c2p * quart + 0.5 * c2 * c2 * quart_p + c2p * Nq + c2 * Nq_p;
        };
        const double g0 = -m[0] * dV;   // dE/ds at s = 0 on the normalised path: -<r, d>
        auto search = [&]() {
            int evals = 0;
            const double s = line_search == OF_LINE_BRENT
                                 ? line_minimum(energy, s_prev, line_tol, evals)
                                 : line_minimum_slope(energy_slope, g0, s_prev, line_tol, evals);
            st.line += evals;
            return s;
        };
        const double tol_line = std::min(1e-5, 1e-2 * st.last_residual);
        prepare_line(tol_line);
        double s = search();
        if (s == 0.0 && tol_line > po.tol) {   // retry with exact line energies
            prepare_line(po.tol);
            s = search();
        }
        if (s == 0.0) break;   // energy flat to rounding along d: stagnated
        const double c = std::sqrt(Ne / (uu + 2.0 * s * ud + s * s * dd));
        launch(k_step, nb, 256, g->stream, n, u, v.d, phi, v.D, v.B, v.C, s, c);
        launch(k_density_plus, nb, 256, g->stream, n, u, v.b, v.rho);
        OF_LAUNCH_CHECK();
        // re-solve (the warm start is nearly exact) to what the next gradient needs: phi's
        // error enters it as 2 u dphi, so a relative accuracy of RESOLVE_FACTOR x the
        // normalised gradient norm keeps that well below the gradient itself; near convergence
        // this reaches the full tolerance, which the final energy and forces use
        KrylovOpts pr = po;
        pr.tol = std::max(po.tol, std::min(1e-6, RESOLVE_FACTOR * st.last_residual));
        poisson_into(g, v.rho, nullptr, phi, pr, st);
        std::swap(v.r, v.rp);
        std::swap(v.d, v.dp);
        rr_prev = rr;
        s_prev = s;
        c_prev = c;
        st.nlcg += 1;
    }
    return converged;
}

// Complex fields of the kernel map's warm starts: one per potential and conjugate pair.
static int lr_ws_fields(const of_functional* fn) {
    return (fn->L == 2 ? 16 : 2) * (fn->n_terms / 2);
}

static void require_conjugate_pairs(const double* P, const double* Q, int n_terms, const char* what) {
    for (int k = 0; k < n_terms; k += 2)
        OF_REQUIRE(P[2 * k] == P[2 * k + 2] && P[2 * k + 1] == -P[2 * k + 3] &&
                       Q[2 * k] == Q[2 * k + 2] && Q[2 * k + 1] == -Q[2 * k + 3],
                   OF_EINVAL, "%s: kernel coefficients %d and %d are not complex conjugates", what, k,
                   k + 1);
}

static void add_info(of_solve_info* out, const of_solve_info& a) {
    if (!out) return;
    out->iterations += a.iterations;
    out->refinements += a.refinements;
    out->net_steps += a.net_steps;
    out->rel_residual = std::max(out->rel_residual, a.rel_residual);
}

// Second-order kernel map (L = 2): the 16 potentials K_mn * u^{2(k+e)} that Eq.
// VLinearResponse:local needs, each the sum of n_terms / 2 shifted solves (one per conjugate
// pair), then V_LR and the T_LR sum from them.  Returns the sum s with T_LR = C_F dV s / 2.
static double lr_potential_l2(of_grid* g, const of_functional* fn, double kf2, const double* u,
                              double* vlr, double* Wws, const KrylovOpts& ko, ScfStats& st,
                              of_solve_info* info_out) {
    const long long n = g->d.n;
    const int nb = vb(n);
    const int npairs = fn->n_terms / 2;
    const double* PC[4] = {fn->P, fn->P10, fn->P20, fn->P11};
    const double* QC[4] = {fn->Q, fn->Q10, fn->Q20, fn->Q11};
    const char* names[4] = {"K_00", "K_10", "K_20", "K_11"};
    for (int c = 0; c < 4; ++c) require_conjugate_pairs(PC[c], QC[c], fn->n_terms, names[c]);
    // class of K_mn (K_mn = K_nm): 00, 10, 20, 11
    auto cls = [](int m, int n_) { return m + n_ == 0 ? 0 : (m == 1 && n_ == 1) ? 3 : m + n_; };
    const double kF = 0.5 * std::sqrt(kf2);
    const double rho_bar = kF * kF * kF / (3.0 * M_PI * M_PI);
    auto fact = [](int k) { return k == 2 ? 2.0 : 1.0; };
    auto binom = [](int m, int p) { return (m == 2 && p == 1) ? 2.0 : 1.0; };
    // the potentials: (class, exponent 0 = alpha / 1 = beta, k), and the coefficient tables
    int pot_of[4][2][3];
    for (auto& a : pot_of) for (auto& b : a) for (int& c : b) c = -1;
    int pot_cls[LR_MAX_POT], pot_e[LR_MAX_POT], pot_k[LR_MAX_POT];
    LrSum S{};
    S.npairs = npairs;
    auto pot = [&](int c, int e, int k) {
        if (pot_of[c][e][k] < 0) {
            OF_REQUIRE(S.npot < LR_MAX_POT, OF_EINVAL, "kernel map: too many potentials");
            pot_of[c][e][k] = S.npot;
            pot_cls[S.npot] = c;
            pot_e[S.npot] = e;
            pot_k[S.npot] = k;
            ++S.npot;
        }
        return pot_of[c][e][k];
    };
    for (int m = 0; m <= 2; ++m)
        for (int nn = 0; m + nn <= 2; ++nn)
            for (int p = 0; p <= m; ++p)
                for (int q = 0; q <= nn; ++q) {
                    // C_mnpq = (-1)^{p+q} / (m! n!) binom(m,p) binom(n,q) rho_bar^{p+q-m-n} (Sec. 2)
                    const double C = ((p + q) % 2 ? -1.0 : 1.0) / (fact(m) * fact(nn)) * binom(m, p) *
                                     binom(nn, q) * std::pow(rho_bar, (double)(p + q - m - nn));
                    const int c = cls(m, nn), ka = m - p, kb = nn - q;
                    const int pb = pot(c, 1, kb), pa = pot(c, 0, ka);
                    // u^{2(m-p+alpha)} V_{mnq beta} and u^{2(n-q+beta)} V_{mnp alpha}
                    S.cv[pb][ka] += C * (ka + fn->alpha);
                    S.ct[pb][ka] += C;
                    S.cv[pa][3 + kb] += C * (kb + fn->beta);
                    S.ct[pa][3 + kb] += C;
                }
    double* scratch = (double*)ws(g, WS_LR, sizeof(double) * 8 * (size_t)n);
    double* gp = scratch;            // six density powers
    double* f00 = scratch + 6 * n;   // -(1/kf2) L_h u^{2 alpha}, -(1/kf2) L_h u^{2 beta}
    launch(k_powers6, nb, 256, g->stream, n, u, 2.0 * fn->alpha, 2.0 * fn->beta, gp);
    OF_LAUNCH_CHECK();
    launch_stencil<double, 2>(g, g->w64, OpScaledLap{gp, f00, -1.0 / kf2});
    launch_stencil<double, 2>(g, g->w64, OpScaledLap{gp + 3 * n, f00 + n, -1.0 / kf2});
    // the solves, one per potential and conjugate pair, two at a time (run_pair)
    const int njobs = S.npot * npairs;
    auto solve = [&](of_grid* h, int job, of_solve_info& si) {
        const int p = job / npairs, r = job % npairs;
        const int c = pot_cls[p], e = pot_e[p], k = pot_k[p];
        // right-hand side: the density power itself, or -(1/kf2) L_h of it for K_00 (Sec. 3.1)
        const double* f = c == 0 ? f00 + (size_t)e * n : gp + (size_t)(3 * e + k) * n;
        const double2 P = make_double2(PC[c][4 * r], PC[c][4 * r + 1]);
        const double2 Q = make_double2(QC[c][4 * r], QC[c][4 * r + 1]);
        double2* W = (double2*)Wws + (size_t)job * n;
        S.W[p][r] = W;
        return shifted(h, f, P, Q, kf2, W, ko, &si);
    };
    for (int job = 0; job < njobs; job += GROUP_MAX) {
        const int k = std::min(GROUP_MAX, njobs - job);
        of_solve_info si[GROUP_MAX] = {};
        of_status sj[GROUP_MAX] = {};
        run_group(g, k, [&](of_grid* h, int q) { sj[q] = solve(h, job + q, si[q]); });
        for (int q = 0; q < k; ++q) {
            if (sj[q] != OF_OK && sj[q] != OF_ENOCONV) throw Error{sj[q]};
            st.kernel += si[q].iterations;
            add_info(info_out, si[q]);
        }
    }
    launch(k_lr_assemble2, nb, 256, g->stream, n, u, (const double*)gp, S, vlr, red_ctx(g, SC_TLR));
    OF_LAUNCH_CHECK();
    return sc(g, SC_TLR);
}

// Kernel map V[u] (Eq. MVF): V_LR into vlr, returns the sum s with T_LR = C_F dV s / 2.
static double lr_potential_impl(of_grid* g, const of_functional* fn, double kf2, const double* u,
                                double* vlr, double* Wws, const KrylovOpts& ko, ScfStats& st,
                                of_solve_info* info_out) {
    const long long n = g->d.n;
    const int nb = vb(n);
    OF_REQUIRE(fn->n_terms >= 2 && fn->n_terms <= 8 && fn->n_terms % 2 == 0, OF_EINVAL,
               "kernel term needs 2..8 coefficients in conjugate pairs (got %d)", fn->n_terms);
    OF_REQUIRE(fn->L == 0 || fn->L == 2, OF_EINVAL, "kernel expansion order L = %d (0 or 2)", fn->L);
    if (fn->L == 2) return lr_potential_l2(g, fn, kf2, u, vlr, Wws, ko, st, info_out);
    require_conjugate_pairs(fn->P, fn->Q, fn->n_terms, "K_00");
    const int npairs = fn->n_terms / 2;
    double* scratch = (double*)ws(g, WS_LR, sizeof(double) * 4 * (size_t)n);
    double *ga = scratch, *gb = scratch + n, *fa = scratch + 2 * n, *fb = scratch + 3 * n;
    launch(k_powers, nb, 256, g->stream, n, u, 2.0 * fn->alpha, 2.0 * fn->beta, ga, gb);
    OF_LAUNCH_CHECK();
    // f_e = -(1/kf2) L u^{2e}  (the m = n = 0 right-hand side of Sec. 3.1)
    launch_stencil<double, 2>(g, g->w64, OpScaledLap{ga, fa, -1.0 / kf2});
    launch_stencil<double, 2>(g, g->w64, OpScaledLap{gb, fb, -1.0 / kf2});
    PairPtrs W{};
    W.npairs = npairs;
    // the shifted solves (two exponents x npairs shifts), up to GROUP_MAX at once on the grid
    // and its twin chain
    const int njobs = 2 * npairs;
    double2* Wj[2 * 4];
    for (int j = 0; j < njobs; ++j) Wj[j] = (double2*)Wws + (size_t)j * n;   // even: u^{2 alpha}
    for (int k = 0; k < npairs; ++k) {
        W.Wa[k] = Wj[2 * k];
        W.Wb[k] = Wj[2 * k + 1];
    }
    for (int job = 0; job < njobs; job += GROUP_MAX) {
        const int kk = std::min(GROUP_MAX, njobs - job);
        of_solve_info si[GROUP_MAX] = {};
        of_status sj[GROUP_MAX] = {};
        run_group(g, kk, [&](of_grid* h, int q) {
            const int j = job + q, k = j / 2;
            const double2 P = make_double2(fn->P[4 * k], fn->P[4 * k + 1]);
            const double2 Q = make_double2(fn->Q[4 * k], fn->Q[4 * k + 1]);
            sj[q] = shifted(h, (j & 1) ? fb : fa, P, Q, kf2, Wj[j], ko, &si[q]);
        });
        for (int q = 0; q < kk; ++q) {
            if (sj[q] != OF_OK && sj[q] != OF_ENOCONV) throw Error{sj[q]};
            st.kernel += si[q].iterations;
            add_info(info_out, si[q]);
        }
    }
    launch(k_lr_assemble, nb, 256, g->stream, n, u, W, fn->alpha, fn->beta, vlr, red_ctx(g, SC_TLR));
    OF_LAUNCH_CHECK();
    return sc(g, SC_TLR);
}

// Small dense solve G x = y (Gaussian elimination, partial pivoting); false if singular.
static bool dense_solve(std::vector<double> G, std::vector<double> y, int m, std::vector<double>& x) {
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(G[i * m + i]));
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(G[r * m + c]) > std::fabs(G[piv * m + c])) piv = r;
        if (!(std::fabs(G[piv * m + c]) > 1e-14 * scale)) return false;
        if (piv != c) {
            for (int k = 0; k < m; ++k) std::swap(G[c * m + k], G[piv * m + k]);
            std::swap(y[c], y[piv]);
        }
        for (int r = c + 1; r < m; ++r) {
            const double f = G[r * m + c] / G[c * m + c];
            for (int k = c; k < m; ++k) G[r * m + k] -= f * G[c * m + k];
            y[r] -= f * y[c];
        }
    }
    x.assign(m, 0.0);
    for (int r = m - 1; r >= 0; --r) {
        double s = y[r];
        for (int k = r + 1; k < m; ++k) s -= G[r * m + k] * x[k];
        x[r] = s / G[r * m + r];
    }
    return true;
}

static void launch_gram(of_grid* g, int m, long long n, const HistPtrs& H, const double* f) {
    const int nb = vb(n);
    switch (m) {
        case 1: launch(k_gram<1>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 2: launch(k_gram<2>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 3: launch(k_gram<3>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 4: launch(k_gram<4>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 5: launch(k_gram<5>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 6: launch(k_gram<6>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        case 7: launch(k_gram<7>, nb, 256, g->stream, n, H, f, red_ctx(g, SC_GRAM)); break;
        default: OF_REQUIRE(false, OF_EINVAL, "Anderson history %d not in 1..7", m);
    }
    OF_LAUNCH_CHECK();
}

// Order-2N FD gradient weights of Eq. gradient:approximate per axis:
// w~_p = (-1)^{p+1} (N!)^2 / (h p (N-p)! (N+p)!), p = 1..N
struct GradWeights {
    double w[3][OF_MAX_N + 1];
    int N;
};

// sum over the grid of |grad_h u|^2, periodic wrap of every index
__global__ void __launch_bounds__(256) k_grad_sq(Dims d, GradWeights G, const double* u, RedCtx rc) {
    double acc[1] = {0.0};
    const long long sz = (long long)d.n1 * d.n2;
    GRID_LOOP(idx, d.n) {
        const int i = (int)(idx % d.n1), j = (int)((idx / d.n1) % d.n2), k = (int)(idx / sz);
        const long long row = (long long)k * sz + (long long)j * d.n1;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int p = 1; p <= G.N; ++p) {
            gx += G.w[0][p] * (u[row + wrap_index(i + p, d.n1)] - u[row + wrap_index(i - p, d.n1)]);
            gy += G.w[1][p] * (u[(long long)k * sz + (long long)wrap_index(j + p, d.n2) * d.n1 + i] -
                               u[(long long)k * sz + (long long)wrap_index(j - p, d.n2) * d.n1 + i]);
            gz += G.w[2][p] * (u[(long long)wrap_index(k + p, d.n3) * sz + (long long)j * d.n1 + i] -
                               u[(long long)wrap_index(k - p, d.n3) * sz + (long long)j * d.n1 + i]);
        }
        acc[0] += gx * gx + gy * gy + gz * gz;
    }
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

static double grad_sq_sum(of_grid* g, const double* u) {
    GradWeights G{};
    G.N = g->N;
    double fN = 1.0;
    for (int q = 2; q <= g->N; ++q) fN *= q;
    for (int a = 0; a < 3; ++a)
        for (int p = 1; p <= g->N; ++p) {
            double den = g->h[a] * p;
            for (int q = 2; q <= g->N - p; ++q) den *= q;   // (N-p)!
            double num = fN * fN;
            for (int q = 2; q <= g->N + p; ++q) num /= q;   // / (N+p)!
            G.w[a][p] = ((p + 1) % 2 ? -1.0 : 1.0) * num / den;
        }
    launch(k_grad_sq, vb(g->d.n), 256, g->stream, g->d, G, u, red_ctx(g, SC_GRADSQ));
    OF_LAUNCH_CHECK();
    return sc(g, SC_GRADSQ);
}

static void energy_terms(of_grid* g, const of_functional* fn, const double* u, const double* b,
                         const double* phi, double t_lr_sum, double e_self, double e_c,
                         int vw_energy, of_scf_result* res) {
    launch_stencil<double, 2>(g, g->w64, OpEnergy{u, b, phi, red_ctx(g, SC_EN)});
    double e[4];
    fetch_scalars(g, SC_EN, 4, e);
    const double dV = g->dV;
    res->e_tf = e[0] * dV;   // e[0] already carries C_F
    // vW: -(lam/2) <u, L_h u> (its gradient is the Hamiltonian's), or (lam/2) int |grad_h u|^2
    res->e_vw = vw_energy == OF_VW_GRADIENT ? 0.5 * fn->lambda * grad_sq_sum(g, u) * dV
                                            : -0.5 * fn->lambda * e[1] * dV;
    res->e_xc = e[2] * dV;
    res->e_es = 0.5 * e[3] * dV;
    res->e_lr = fn->mu != 0.0 ? fn->mu * 0.5 * OF_CF * t_lr_sum * dV : 0.0;
    res->e_self = e_self;
    res->e_corr = e_c;
    res->energy = res->e_tf + res->e_vw + res->e_lr + res->e_xc + res->e_es + res->e_self + res->e_corr;
}

static void scf(of_grid* g, const of_system* sys, const of_functional* fn, const of_scf_opts* o,
                double* u, double* phi, of_scf_result* res) {
    const long long n = g->d.n;
    const int nb = vb(n);
    const double dV = g->dV;
    double Ne = 0.0;
    for (int J = 0; J < sys->n_atoms; ++J) Ne += sys->Z[J];
    OF_REQUIRE(Ne > 0, OF_EINVAL, "total ionic charge must be positive");
    const FnParams fp = fn_params(fn);
    const bool lr = fn->mu != 0.0;
    KrylovOpts po = krylov_opts(&o->poisson), ko = krylov_opts(&o->kernel);
    if (o->precision == OF_F32) po.precision = ko.precision = OF_F32;

    ScfVecs v = scf_vecs(g);
    std::memset(res, 0, sizeof(*res));
    OF_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * n, g->stream));
    double e_self = 0.0, e_c = 0.0;
    pseudocharge(g, sys, v.b, &e_self);
    overlap_correction(g, sys, &e_c, nullptr);
    ScfStats st;
    OF_CUDA(cudaMemsetAsync(v.D, 0, sizeof(double) * n, g->stream));
    poisson_into(g, v.b, nullptr, v.D, po, st);   // phi_b
    for (double* p : {v.B, v.C, v.V, v.rp, v.dp})
        OF_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * n, g->stream));

    const double kf = std::cbrt(3.0 * M_PI * M_PI * Ne / (g->L[0] * g->L[1] * g->L[2]));
    const double kf2 = 4.0 * kf * kf;
    const int m = std::max(0, std::min(o->anderson_m, 7));
    double* Wws = nullptr;
    double *Shist = nullptr, *Yhist = nullptr, *Vprev = nullptr, *fcur = nullptr, *fprev = nullptr;
    if (lr) {
        // Anderson history (S, Y), V_{k-1}, f_k, f_{k-1}, then the kernel-solve warm starts
        double* hist = (double*)ws(g, WS_AND, sizeof(double) * (size_t)n * (2 * m + 3 + 2 * lr_ws_fields(fn)));
        Shist = hist;
        Yhist = hist + (size_t)m * n;
        Vprev = hist + (size_t)2 * m * n;
        fcur = Vprev + n;
        fprev = fcur + n;
        Wws = fprev + n;   // lr_ws_fields complex fields
        OF_CUDA(cudaMemsetAsync(Wws, 0, sizeof(double2) * n * lr_ws_fields(fn), g->stream));
    }

    double t_lr_sum = 0.0;
    int hist_count = 0, hist_head = 0;
    double err = 0.0;
    bool inner_ok = true;
    double prev_err = 1.0;
    // fixed point on u instead of V_LR (Sec. 5.3, Table MixComparison): the mixed iterate is
    // u_k (kept in v.Vhat), the map u_k -> U(V[u_k])
    const bool fp_u = lr && o->fixed_point == OF_FP_U;
    double* xk = fp_u ? v.Vhat : v.V;   // the iterate Anderson mixes
    for (int k = 0; k < std::max(1, o->fp_max_iter); ++k) {
        // inexact inner solves while the outer iteration is far from its fixed point
        const double tol_k = (lr && o->nlcg_tol_rel > 0.0)
                                 ? std::max(o->nlcg_tol, o->nlcg_tol_rel * prev_err)
                                 : o->nlcg_tol;
        // the kernel map's tolerance: 1e-2 of the previous fixed-point error, at most 1e-5
        KrylovOpts kk = ko;
        kk.tol = std::max(ko.tol, std::min(1e-5, 1e-2 * prev_err));
        if (fp_u) {
            // u_k normalised to N_e (mixing does not keep the norm), V = V[u_k], u_k kept
            launch(k_sum_product, nb, 256, g->stream, n, u, u, red_ctx(g, SC_UU));
            OF_LAUNCH_CHECK();
            const double uu = sc(g, SC_UU) * dV;
            OF_REQUIRE(uu > 0 && std::isfinite(uu), OF_EBREAKDOWN, "fixed point on u: iterate has norm %g", uu);
            launch(k_scale, nb, 256, g->stream, n, u, std::sqrt(Ne / uu));
            OF_LAUNCH_CHECK();
            t_lr_sum = lr_potential_impl(g, fn, kf2, u, v.V, Wws, kk, st, nullptr);
            OF_CUDA(cudaMemcpyAsync(xk, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
        }
        inner_ok = nlcg(g, fp, Ne, v, u, phi, lr ? v.V : nullptr, tol_k, o->nlcg_max_iter,
                        std::max(1, o->nlcg_restart), o->line_tol > 0 ? o->line_tol : 1e-3,
                        o->line_search, po, st, o->nlcg_precond_shift, o->nlcg_precond_low);
        res->outer_iterations = k + 1;
        if (!lr) { err = 0.0; break; }
        if (fp_u) {
            // f = U(V[u_k]) - u_k
            launch(k_fp_residual, nb, 256, g->stream, n, (const double*)u, (const double*)xk, fcur,
                   red_ctx(g, SC_FP));
        } else {
            // inexact kernel map while the fixed point is far off (the shifted solves stop at
            // 1e-3 of the previous fixed-point error, at most 1e-6, never below the requested
            // tolerance); the converged map is evaluated to ~1e-9.  f = V[u_k] - V_k
            t_lr_sum = lr_potential_impl(g, fn, kf2, u, v.Vhat, Wws, kk, st, nullptr);
            launch(k_fp_residual, nb, 256, g->stream, n, v.Vhat, v.V, fcur, red_ctx(g, SC_FP));
        }
        OF_LAUNCH_CHECK();
        double nf[2];
        fetch_scalars(g, SC_FP, 2, nf);
        err = nf[1] > 0 ? std::sqrt(nf[0] / nf[1]) : 0.0;
        prev_err = err;
        if (o->verbose)
            fprintf(stderr, "[of] outer %d: fp error %.3e, nlcg %d, poisson its %d, kernel its %d\n",
                    k, err, st.nlcg, st.poisson, st.kernel);
        if (err < o->fp_tol && tol_k <= o->nlcg_tol) break;
        if (k + 1 >= o->fp_max_iter) break;
        // history: S = x_k - x_{k-1}, Y = f_k - f_{k-1} (x = V_LR, or u)
        if (k > 0 && m > 0) {
            const int slot = hist_head;
            launch(k_diff, nb, 256, g->stream, n, xk, Vprev, Shist + (size_t)slot * n);
            launch(k_diff, nb, 256, g->stream, n, fcur, fprev, Yhist + (size_t)slot * n);
            OF_LAUNCH_CHECK();
            hist_head = (hist_head + 1) % m;
            hist_count = std::min(hist_count + 1, m);
        }
        OF_CUDA(cudaMemcpyAsync(Vprev, xk, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
        OF_CUDA(cudaMemcpyAsync(fprev, fcur, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
        HistPtrs H{};
        int j = hist_count;
        std::vector<double> gamma;
        while (j > 0) {
            // use the j most recent columns, oldest first
            H.m = j;
            for (int a = 0; a < j; ++a) {
                const int slot = ((hist_head - j + a) % m + m) % m;
                H.S[a] = Shist + (size_t)slot * n;
                H.Y[a] = Yhist + (size_t)slot * n;
            }
            launch_gram(g, j, n, H, fcur);
            const int K = j * (j + 1) / 2 + j;
            std::vector<double> raw(K);
            fetch_scalars(g, SC_GRAM, K, raw.data());
            std::vector<double> G(j * j), y(j);
            int idx = 0;
            for (int a = 0; a < j; ++a)
                for (int b = a; b < j; ++b) { G[a * j + b] = G[b * j + a] = raw[idx]; ++idx; }
            for (int a = 0; a < j; ++a) y[a] = raw[idx++];
            if (dense_solve(G, y, j, gamma)) break;
            --j;   // drop the oldest column and retry
        }
        H.m = j;
        for (int a = 0; a < j; ++a) H.g[a] = gamma[a];
        launch(k_anderson_update, nb, 256, g->stream, n, xk, fcur, o->anderson_zeta, H);
        OF_LAUNCH_CHECK();
        if (fp_u) OF_CUDA(cudaMemcpyAsync(u, xk, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
    }
    // u-mixing ends on u = U(V[u_k]); its own T_LR for the energy
    if (fp_u) t_lr_sum = lr_potential_impl(g, fn, kf2, u, v.Vhat, Wws, ko, st, nullptr);
    energy_terms(g, fn, u, v.b, phi, t_lr_sum, e_self, e_c, o->vw_energy, res);
    res->fp_error = err;
    res->nlcg_residual = st.last_residual;
    res->nlcg_iterations = st.nlcg;
    res->poisson_iterations = st.poisson;
    res->kernel_iterations = st.kernel;
    res->line_evaluations = st.line;
    res->converged = (inner_ok && (!lr || err < o->fp_tol)) ? 1 : 0;
    (void)dV;
}

}  // namespace of

using namespace of;

extern "C" {

void of_default_scf_opts(of_scf_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nlcg_tol = 1e-7;
    o->nlcg_max_iter = 5000;
    o->nlcg_restart = 50;
    o->fp_tol = 1e-7;
    o->fp_max_iter = 60;
    o->anderson_m = 7;
    o->anderson_zeta = 0.3;
    o->precision = OF_F64;
    of_default_solve_opts(&o->poisson);
    of_default_solve_opts(&o->kernel);
    o->verbose = 0;
    o->line_tol = 1e-3;
    o->line_search = OF_LINE_SLOPE;
}

of_status of_hamiltonian_apply(of_grid* g, const of_functional* fn, const double* u,
                               const double* phi, const double* vlr, double* hu) {
    if (!g || !fn || !u || !phi || !hu || (fn->mu != 0.0 && !vlr)) {
        set_error("of_hamiltonian_apply: null argument");
        return OF_EINVAL;
    }
    try {
        launch_stencil<double, 2>(g, g->w64,
                                  OpHamiltonian{u, phi, fn->mu != 0.0 ? vlr : nullptr, hu, nullptr,
                                                fn_params(fn), red_ctx(g, SC_UHU)});
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

int of_lr_workspace_fields(const of_functional* fn) { return fn ? lr_ws_fields(fn) : 0; }

of_status of_lr_potential(of_grid* g, const of_functional* fn, double kf2, const double* u,
                          double* vlr, double* t_lr, double* W_ws, const of_solve_opts* opts,
                          of_solve_info* info) {
    if (!g || !fn || !u || !vlr || !(kf2 > 0)) { set_error("of_lr_potential: bad argument"); return OF_EINVAL; }
    try {
        if (info) std::memset(info, 0, sizeof(*info));
        double* W = W_ws;
        if (!W) {
            const size_t bytes = sizeof(double2) * (size_t)lr_ws_fields(fn) * g->d.n;
            W = (double*)ws(g, WS_AND, bytes);
            OF_CUDA(cudaMemsetAsync(W, 0, bytes, g->stream));
        }
        ScfStats st;
        const double s = lr_potential_impl(g, fn, kf2, u, vlr, W, krylov_opts(opts), st, info);
        if (t_lr) *t_lr = 0.5 * OF_CF * s * g->dV;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_scf_ground_state_batched(int ncells, of_grid* const* grids, const of_system* systems,
                                      const of_functional* fn, const of_scf_opts* opts,
                                      double* const* u, double* const* phi, of_scf_result* results) {
    if (ncells < 1 || !grids || !systems || !fn || !u || !phi || !results) {
        set_error("of_scf_ground_state_batched: bad argument");
        return OF_EINVAL;
    }
    try {
        for (int c = 0; c < ncells; ++c) {
            OF_REQUIRE(grids[c] && u[c] && phi[c], OF_EINVAL,
                       "of_scf_ground_state_batched: null grid or field for cell %d", c);
            OF_REQUIRE(grids[c]->stream == grids[0]->stream && grids[c]->device == grids[0]->device,
                       OF_EINVAL, "of_scf_ground_state_batched: cell %d differs in stream or device", c);
            for (int k = 0; k < c; ++k)
                OF_REQUIRE(grids[k] != grids[c], OF_EINVAL,
                           "of_scf_ground_state_batched: cells %d and %d share a grid handle", k, c);
        }
        of_scf_opts o;
        if (opts) o = *opts; else of_default_scf_opts(&o);
        return run_on_stream_pool(ncells, grids, [&](int c) -> of_status {
            scf(grids[c], &systems[c], fn, &o, u[c], phi[c], &results[c]);
            if (!results[c].converged) {
                set_error("ground state not converged: nlcg residual %.3e, fixed-point error %.3e",
                          results[c].nlcg_residual, results[c].fp_error);
                return OF_ENOCONV;
            }
            return OF_OK;
        });
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

void of_default_relax_opts(of_relax_opts* o) {
    if (!o) return;
    o->ftol = 1e-3;
    o->max_steps = 40;
    o->step0 = 0.05;
    o->line_tol = 0.1;
    o->max_line = 4;
}

// Geometry relaxation (Sec. 3.3): NLCG on the positions of sys's ions (Polak-Ribiere, restarted
// at beta < 0 or an uphill direction) with a secant line search on E'(s) = -F . d.  Every
// evaluation is a ground state warm-started from u, then the forces.  R_out (host, 3 n_atoms):
// final positions; F_out (may be null): final forces; e_first (may be null): the ground-state
// energy at the starting positions.  Throws Error; res->converged tells whether max |F| < ftol.
static void relax_impl(of_grid* g, const of_system* sys, const of_functional* fn,
                       const of_scf_opts& so, const of_relax_opts& ro, double* u, double* phi,
                       double* R_out, double* F_out, of_relax_result* res, double* e_first) {
    {
        std::memset(res, 0, sizeof(*res));
        const size_t m3 = 3 * (size_t)sys->n_atoms;
        std::vector<double> R(sys->R, sys->R + m3), F(m3), Fp(m3), d(m3), Rs(m3), Fs(m3);
        of_system sx = *sys;
        of_scf_result gs{};
        auto dot = [&](const std::vector<double>& a, const std::vector<double>& b) {
            double s = 0.0;
            for (size_t i = 0; i < m3; ++i) s += a[i] * b[i];
            return s;
        };
        auto maxabs = [&](const std::vector<double>& a) {
            double s = 0.0;
            for (double v : a) s = std::max(s, std::fabs(v));
            return s;
        };
        // ground state (warm-started from u) and forces at positions Rx
        auto evaluate = [&](const std::vector<double>& Rx, std::vector<double>& Fx) {
            sx.R = Rx.data();
            scf(g, &sx, fn, &so, u, phi, &gs);
            ++res->evaluations;
            OF_REQUIRE(gs.converged, OF_ENOCONV,
                       "of_relax: ground state %d not converged (nlcg residual %.3e, fixed-point error %.3e)",
                       res->evaluations, gs.nlcg_residual, gs.fp_error);
            forces(g, &sx, phi, Fx.data());
        };
        evaluate(R, F);
        if (e_first) *e_first = gs.energy;
        d = F;
        bool have_prev = false;
        while (res->steps < ro.max_steps && maxabs(F) >= ro.ftol) {
            if (have_prev) {   // Polak-Ribiere, restarted at beta < 0
                double num = 0.0;
                for (size_t i = 0; i < m3; ++i) num += F[i] * (F[i] - Fp[i]);
                const double beta = std::max(0.0, num / dot(Fp, Fp));
                for (size_t i = 0; i < m3; ++i) d[i] = F[i] + beta * d[i];
            }
            double g0 = -dot(F, d);   // E'(0) along d
            if (!(g0 < 0.0)) {        // not downhill: restart along F
                d = F;
                g0 = -dot(F, F);
            }
            double sa = 0.0, ga = g0, s = ro.step0 / maxabs(d);
            for (int j = 0; j < ro.max_line; ++j) {
                for (size_t i = 0; i < m3; ++i) Rs[i] = R[i] + s * d[i];
                evaluate(Rs, Fs);
                const double gv = -dot(Fs, d);
                if (std::fabs(gv) <= ro.line_tol * std::fabs(g0) || j + 1 == ro.max_line) break;
                // secant root of E'(s) through the last two points; without positive curvature
                // seen yet, a longer step
                const double sn = gv > ga ? s - gv * (s - sa) / (gv - ga) : 2.0 * s;
                sa = s;
                ga = gv;
                s = sn;
            }
            Fp = F;
            R = Rs;
            F = Fs;
            have_prev = true;
            ++res->steps;
        }
        res->energy = gs.energy;
        res->max_force = maxabs(F);
        res->converged = res->max_force < ro.ftol;
        std::copy(R.begin(), R.end(), R_out);
        if (F_out) std::copy(F.begin(), F.end(), F_out);
    }
}

static void check_relax_opts(const of_relax_opts& ro, const char* where) {
    OF_REQUIRE(ro.ftol > 0 && ro.step0 > 0 && ro.max_line >= 1 && ro.max_steps >= 0, OF_EINVAL,
               "%s: bad relaxation options", where);
}

of_status of_relax(of_grid* g, const of_system* sys, const of_functional* fn,
                   const of_scf_opts* scf_opts, const of_relax_opts* opts, double* u, double* phi,
                   double* R_out, double* F_out, of_relax_result* res) {
    if (!g || !sys || !sys->R || sys->n_atoms < 1 || !fn || !u || !phi || !R_out || !res) {
        set_error("of_relax: null argument");
        return OF_EINVAL;
    }
    try {
        of_scf_opts so;
        if (scf_opts) so = *scf_opts; else of_default_scf_opts(&so);
        of_relax_opts ro;
        if (opts) ro = *opts; else of_default_relax_opts(&ro);
        check_relax_opts(ro, "of_relax");
        relax_impl(g, sys, fn, so, ro, u, phi, R_out, F_out, res, nullptr);
        if (!res->converged) {
            set_error("of_relax: max force %.3e after %d steps", res->max_force, res->steps);
            return OF_ENOCONV;
        }
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

// Vacancy formation energy (Sec. 5.6): E_vf = E(M-1, 1, (M-1)/M Omega) - ((M-1)/M) E(M, 0, Omega).
// The vacancy cell keeps the volume per atom: its sides and the remaining positions are the
// perfect cell's scaled by ((M-1)/M)^{1/3} about the origin, on the same number of grid points.
// The two cells' ground states run at once on the stream pool; the vacancy cell's relaxation
// (optional) follows its own ground state.
of_status of_vacancy_formation(of_grid* perfect, of_grid* vacancy, const of_system* sys, int site,
                               const of_functional* fn, const of_scf_opts* scf_opts,
                               const of_relax_opts* relax_opts, double* u_perfect,
                               double* phi_perfect, double* u_vacancy, double* phi_vacancy,
                               double* R_out, of_vacancy_result* res) {
    if (!perfect || !vacancy || !sys || !sys->R || !sys->Z || !fn || !u_perfect || !phi_perfect ||
        !u_vacancy || !phi_vacancy || !res) {
        set_error("of_vacancy_formation: null argument");
        return OF_EINVAL;
    }
    try {
        const int M = sys->n_atoms;
        OF_REQUIRE(M >= 2 && site >= 0 && site < M, OF_EINVAL,
                   "of_vacancy_formation: site %d of a cell with %d ions", site, M);
        OF_REQUIRE(perfect != vacancy, OF_EINVAL, "of_vacancy_formation: the two cells share a grid handle");
        OF_REQUIRE(perfect->d.n1 == vacancy->d.n1 && perfect->d.n2 == vacancy->d.n2 &&
                       perfect->d.n3 == vacancy->d.n3 && perfect->N == vacancy->N,
                   OF_EINVAL, "of_vacancy_formation: the vacancy grid must have the perfect grid's "
                   "points (%d x %d x %d) and order", perfect->d.n1, perfect->d.n2, perfect->d.n3);
        OF_REQUIRE(perfect->stream == vacancy->stream && perfect->device == vacancy->device, OF_EINVAL,
                   "of_vacancy_formation: the two handles differ in stream or device");
        const double scale = std::cbrt((double)(M - 1) / (double)M);
        for (int a = 0; a < 3; ++a)
            OF_REQUIRE(std::fabs(vacancy->L[a] - scale * perfect->L[a]) <= 1e-12 * perfect->L[a],
                       OF_EINVAL, "of_vacancy_formation: vacancy cell side %d is %.15g, expected "
                       "((M-1)/M)^(1/3) x %.15g = %.15g", a, vacancy->L[a], perfect->L[a],
                       scale * perfect->L[a]);
        of_scf_opts so;
        if (scf_opts) so = *scf_opts; else of_default_scf_opts(&so);
        of_relax_opts ro;
        if (relax_opts) {
            ro = *relax_opts;
            check_relax_opts(ro, "of_vacancy_formation");
        }
        std::memset(res, 0, sizeof(*res));
        std::vector<double> Rv, Zv;
        for (int J = 0; J < M; ++J) {
            if (J == site) continue;
            for (int c = 0; c < 3; ++c) Rv.push_back(scale * sys->R[3 * J + c]);
            Zv.push_back(sys->Z[J]);
        }
        of_system vs = *sys;
        vs.n_atoms = M - 1;
        vs.R = Rv.data();
        vs.Z = Zv.data();
        std::vector<double> Rfin(Rv), Ffin(Rv.size());
        of_scf_result rp{};
        of_grid* grids[2] = {perfect, vacancy};
        const of_status st = run_on_stream_pool(2, grids, [&](int c) -> of_status {
            if (c == 0) {
                scf(perfect, sys, fn, &so, u_perfect, phi_perfect, &rp);
                OF_REQUIRE(rp.converged, OF_ENOCONV, "perfect cell: ground state not converged "
                           "(nlcg residual %.3e, fixed-point error %.3e)", rp.nlcg_residual, rp.fp_error);
                return OF_OK;
            }
            if (relax_opts) {
                of_relax_result rr{};
                relax_impl(vacancy, &vs, fn, so, ro, u_vacancy, phi_vacancy, Rfin.data(), Ffin.data(),
                           &rr, &res->e_unrelaxed);
                res->e_relaxed = rr.energy;
                res->max_force = rr.max_force;
                res->relax_steps = rr.steps;
                res->evaluations = rr.evaluations;
                OF_REQUIRE(rr.converged, OF_ENOCONV, "vacancy cell: max force %.3e after %d "
                           "relaxation steps", rr.max_force, rr.steps);
            } else {
                of_scf_result rv{};
                scf(vacancy, &vs, fn, &so, u_vacancy, phi_vacancy, &rv);
                OF_REQUIRE(rv.converged, OF_ENOCONV, "vacancy cell: ground state not converged "
                           "(nlcg residual %.3e, fixed-point error %.3e)", rv.nlcg_residual, rv.fp_error);
                forces(vacancy, &vs, phi_vacancy, Ffin.data());
                res->e_unrelaxed = res->e_relaxed = rv.energy;
                for (double f : Ffin) res->max_force = std::max(res->max_force, std::fabs(f));
                res->evaluations = 1;
            }
            return OF_OK;
        });
        const double frac = (double)(M - 1) / (double)M;
        res->e_perfect = rp.energy;
        res->evf_unrelaxed = res->e_unrelaxed - frac * rp.energy;
        res->evf_relaxed = res->e_relaxed - frac * rp.energy;
        if (R_out) std::copy(Rfin.begin(), Rfin.end(), R_out);
        return st;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_scf_ground_state(of_grid* g, const of_system* sys, const of_functional* fn,
                              const of_scf_opts* opts, double* u, double* phi,
                              of_scf_result* res) {
    if (!g || !sys || !fn || !u || !phi || !res) {
        set_error("of_scf_ground_state: null argument");
        return OF_EINVAL;
    }
    try {
        of_scf_opts o;
        if (opts) o = *opts; else of_default_scf_opts(&o);
        scf(g, sys, fn, &o, u, phi, res);
        if (!res->converged) {
            set_error("ground state not converged: nlcg residual %.3e, fixed-point error %.3e",
                      res->nlcg_residual, res->fp_error);
            return OF_ENOCONV;
        }
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

}  // extern "C"
