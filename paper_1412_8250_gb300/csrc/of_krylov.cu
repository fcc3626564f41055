// Krylov solvers driven by the FD Laplacian.
//
//  * Poisson (Eq. Poisson): -(1/4pi) L_h phi = rho, i.e. A phi = 4 pi (rho - mean rho) with
//    A = -L_h symmetric positive semi-definite; CG on the mean-free subspace (the paper uses
//    GMRES; CG is the natural choice for this SPD operator).
//  * Shifted (Eqs. Helmholtz:beta / Helmholtz:alpha): (-(1/kf2) L_h + Q) W = P f with complex
//    Q: the matrix is complex symmetric (A^T = A), so COCG (CG with the bilinear form r^T r)
//    is used in place of the paper's GMRES on the real/imaginary split.
//
// Both run either in FP64, or as iterative refinement: an FP64 residual, an FP32 Krylov
// solve of the correction to a loose relative tolerance, an FP64 update -- repeated until the
// true FP64 residual meets the tolerance.
//
// Every iteration is two kernels: the stencil sweep forms p = r + beta p on the fly (halo
// points included), writes p and A p and reduces p^T A p; the update kernel applies alpha,
// updates x and r and reduces r^T r and |r|^2.  alpha, beta and the stopping flag live in
// device memory, so the host only synchronises every `check_every` iterations.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "of_ff.cuh"
#include "of_krylov.cuh"

namespace of {

// Projected PCG on the singular periodic operator: the preconditioned vector is used with its
// mean removed (z - zbar, zbar = mean z), so rounding in the constant mode, which the
// preconditioner amplifies, never enters the search direction.
// rho_new = r^T (z - zbar) ; beta = rho_new / rho (0 on the first call) ; rho = rho_new.
__global__ void __launch_bounds__(256) k_pcg_beta(long long n, const float* __restrict__ r,
                                                  const float* __restrict__ z, bool first,
                                                  KState* st, RedCtx rc) {
    pdl_enter();
    if (st->done != 0.0) return;
    float prz = 0.f, pz = 0.f, pr = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float ri = r[i], zi = z[i];
        prz += ri * zi;
        pz += zi;
        pr += ri;
    }
    double acc[3] = {(double)prz, (double)pz, (double)pr};
    if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0)
        pcg_finish(st, acc, n, first);
}

// Preconditioned COCG (complex symmetric A, real symmetric positive M): the bilinear form
// rho_new = r^T z (no conjugation) ; beta = rho_new / rho (0 on the first call) ; rho = rho_new.
__global__ void __launch_bounds__(256) k_pcocg_beta(long long n, const float2* __restrict__ r,
                                                    const float2* __restrict__ z, bool first,
                                                    KState* st, RedCtx rc) {
    pdl_enter();
    if (st->done != 0.0) return;
    float pre = 0.f, pim = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 ri = r[i], zi = z[i];
        pre = fmaf(ri.x, zi.x, fmaf(-ri.y, zi.y, pre));
        pim = fmaf(ri.x, zi.y, fmaf(ri.y, zi.x, pim));
    }
    double acc[2] = {(double)pre, (double)pim};
    if (grid_reduce<2>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0)
        pcocg_finish(st, acc, first);
}

// ---------------------------------------------------------------- small vector kernels
// sum of a[i] * (b ? b[i] : 1) over the grid into out[0]
__global__ void __launch_bounds__(256) k_sum_product(long long n, const double* a, const double* b,
                                                     RedCtx rc) {
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc[0] += b ? a[i] * b[i] : a[i];
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

// y = scale * (a*b - mean), mean = *sum_dev / n ; b may be null (then a alone)
__global__ void k_form_rhs(long long n, const double* a, const double* b, const double* sum_dev,
                           double scale, double* y) {
    const double mean = *sum_dev / (double)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = scale * ((b ? a[i] * b[i] : a[i]) - mean);
}

__global__ void k_sub_mean(long long n, double* x, const double* sum_dev) {
    const double mean = *sum_dev / (double)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] -= mean;
}

// complex rhs b = P f
__global__ void k_scale_complex(long long n, const double* f, double2 P, double2* b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = make_double2(P.x * f[i], P.y * f[i]);
}

// |b|^2 into state tol2 (times tol^2) -- Hermitian norm of a real or complex field
template <typename T>
__global__ void __launch_bounds__(256) k_norm_to_tol(long long n, const T* b, double tol,
                                                     KState* st, RedCtx rc) {
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc[0] += hn2(b[i]);
    if (grid_reduce<1>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->tol2 = tol * tol * acc[0];
        st->red[1] = acc[0];
    }
}

// FP64 residual -> FP32 right-hand side; fresh inner state with rr, r^T r in FP64
template <typename T64, typename T32>
__global__ void __launch_bounds__(256) k_demote(long long n, const T64* r64, T32* r32, T32* e32,
                                                double inner_tol, const KState* outer, KState* st,
                                                int maxit, RedCtx rc);

template <>
__global__ void __launch_bounds__(256) k_demote<double, float>(long long n, const double* r64, float* r32,
                                                               float* e32, double inner_tol,
                                                               const KState* outer, KState* st,
                                                               int maxit, RedCtx rc) {
    // the residual is scaled to unit RMS before rounding, so tiny right-hand sides (near the
    // end of a minimisation) stay inside the FP32 normal range
    const double inv = outer->rr > 0.0 ? rsqrt(outer->rr / (double)n) : 1.0;
    float part = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(r64[i] * inv);
        r32[i] = v;
        e32[i] = 0.0f;
        part += v * v;
    }
    double acc[3] = {(double)part, (double)part, 0.0};
    if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->rr = acc[0];
        st->rho_re = acc[0];
        st->rho_im = 0.0;
        st->scale = 1.0 / inv;
        st->tol2 = inner_tol * inner_tol * acc[0];
        st->beta_re = st->beta_im = 0.0;
        st->done = (acc[0] <= st->tol2) ? 1.0 : 0.0;
        st->iters = 0.0;
        st->maxit = maxit;
        st->breakdown = 0.0;
        st->zshift = 0.0;
    }
}

template <>
__global__ void __launch_bounds__(256) k_demote<double2, float2>(long long n, const double2* r64,
                                                                 float2* r32, float2* e32,
                                                                 double inner_tol,
                                                                 const KState* outer, KState* st,
                                                                 int maxit, RedCtx rc) {
    const double inv = outer->rr > 0.0 ? rsqrt(outer->rr / (double)n) : 1.0;
    float p0 = 0.f, p1 = 0.f, p2 = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = make_float2((float)(r64[i].x * inv), (float)(r64[i].y * inv));
        r32[i] = v;
        e32[i] = make_float2(0.0f, 0.0f);
        p0 += hn2f(v);
        const float2 s = bilf(v, v);
        p1 += s.x;
        p2 += s.y;
    }
    double acc[3] = {(double)p0, (double)p1, (double)p2};
    if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->rr = acc[0];
        st->rho_re = acc[1];
        st->rho_im = acc[2];
        st->scale = 1.0 / inv;
        st->tol2 = inner_tol * inner_tol * acc[0];
        st->beta_re = st->beta_im = 0.0;
        st->done = (acc[0] <= st->tol2) ? 1.0 : 0.0;
        st->iters = 0.0;
        st->maxit = maxit;
        st->breakdown = 0.0;
        st->zshift = 0.0;
    }
}

__device__ __forceinline__ void add_promoted(double& x, float e, double s) { x += s * (double)e; }
__device__ __forceinline__ void add_promoted(double2& x, float2 e, double s) {
    x.x += s * (double)e.x;
    x.y += s * (double)e.y;
}
// x += scale * e, scale the factor the inner right-hand side was divided by
template <typename T64, typename T32>
__global__ void k_promote_add(long long n, T64* x, const T32* e, const KState* inner) {
    const double s = inner->scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        add_promoted(x[i], e[i], s);
}

__global__ void k_init_state(KState* st, int maxit) {
    st->zshift = 0.0;
    st->iters = 0.0;
    st->maxit = maxit;
    st->done = 0.0;
    st->breakdown = 0.0;
}

// ---------------------------------------------------------------- host drivers
KrylovOpts krylov_opts(const of_solve_opts* o) {
    KrylovOpts k{1e-10, 20000, OF_F64, 1e-5, 8, 0, nullptr, 0.3};
    if (o) {
        k.no_multigrid = o->no_multigrid;
        k.precond = o->precond;
        if (o->precond_theta > 0) k.theta = o->precond_theta;
        if (o->tol > 0) k.tol = o->tol;
        if (o->max_iter > 0) k.max_iter = o->max_iter;
        k.precision = o->precision;
        if (o->inner_tol > 0) k.inner_tol = o->inner_tol;
        if (o->check_every > 0) k.check_every = o->check_every;
    }
    return k;
}

static void pcg_init_body(of_grid* g, float* r, float* z, KState* st) {
    const long long n = g->d.n;
    if (mg_vcycle_beta(g, r, z, st, true)) return;
    ProfScope ps(g, PC_UPDATE, 2.0 * sizeof(float) * (double)n);
    launch_pdl(k_pcg_beta, vec_blocks(n), 256, 0, g->stream, n, r, z, true, st, red_ctx(g, 0));
}

static void pcg_step_body(of_grid* g, float* x, float* r, float* pin, float* pout, float* Ap,
                          float* z, KState* st) {
    const long long n = g->d.n;
    OpKrylovA<float> op{z, pin, pout, Ap, st, red_ctx(g, 0), 1.0f, make_double2(0.0, 0.0)};
    launch_stencil<float, 2>(g, g->w32, op);
    {
        ProfScope ps(g, PC_UPDATE, 6.0 * sizeof(float) * (double)n);
        launch_krylov_update<float, true>(g, n, x, r, pout, Ap, st, red_ctx(g, 0), vec_blocks(n));
    }
    if (mg_vcycle_beta(g, r, z, st, false)) return;
    ProfScope ps(g, PC_UPDATE, 2.0 * sizeof(float) * (double)n);
    launch_pdl(k_pcg_beta, vec_blocks(n), 256, 0, g->stream, n, r, z, false, st, red_ctx(g, 0));
}

static void pcocg_init_body(of_grid* g, float2* r, float2* z, KState* st, double sigma) {
    const long long n = g->d.n;
    if (mg_vcycle_shifted_beta(g, r, z, st, true, sigma)) return;
    ProfScope ps(g, PC_UPDATE, 2.0 * sizeof(float2) * (double)n);
    launch_pdl(k_pcocg_beta, vec_blocks(n), 256, 0, g->stream, n, (const float2*)r, (const float2*)z,
               true, st, red_ctx(g, 0));
}

static void pcocg_step_body(of_grid* g, float2* x, float2* r, float2* pin, float2* pout, float2* Ap,
                            float2* z, KState* st, float a, double2 Q, double sigma) {
    const long long n = g->d.n;
    OpKrylovA<float2> op{z, pin, pout, Ap, st, red_ctx(g, 0), a, Q};
    launch_stencil<float2, 1>(g, g->w32, op);
    {
        ProfScope ps(g, PC_UPDATE, 6.0 * sizeof(float2) * (double)n);
        launch_krylov_update<float2, true>(g, n, x, r, pout, Ap, st, red_ctx(g, 0), vec_blocks(n));
    }
    if (mg_vcycle_shifted_beta(g, r, z, st, false, sigma)) return;
    ProfScope ps(g, PC_UPDATE, 2.0 * sizeof(float2) * (double)n);
    launch_pdl(k_pcocg_beta, vec_blocks(n), 256, 0, g->stream, n, (const float2*)r, (const float2*)z,
               false, st, red_ctx(g, 0));
}

// One plain CG / COCG iteration: p_out = r + beta p_in with A p_out and p^T A p in one sweep,
// then the update of x and r with the next beta.
template <typename T>
static void krylov_step(of_grid* g, KState* st, T* x, T* r, T* pin, T* pout, T* Ap,
                        typename KT<T>::R a, double2 Q, const Weights<typename KT<T>::R>& W) {
    const long long n = g->d.n;
    constexpr int RY = KT<T>::cplx ? 1 : 2;
    OpKrylovA<T> op{r, pin, pout, Ap, st, red_ctx(g, 0), a, Q};
    launch_stencil<T, RY>(g, W, op);
    ProfScope ps(g, PC_UPDATE, 6.0 * sizeof(T) * (double)n);
    launch_krylov_update<T, false>(g, n, x, r, pout, Ap, st, red_ctx(g, 0), vec_blocks(n));
}

// Runs Krylov iterations on state `st` until its done flag is set.  Returns host copy.  Pairs
// of iterations (ping and pong of the direction buffers) are replayed from a cached CUDA graph
// keyed by the buffers and the operator's constants.
template <typename T>
static KState iterate(of_grid* g, int st_off, T* x, T* r, T* pa, T* pb, T* Ap,
                      typename KT<T>::R a, double2 Q, const Weights<typename KT<T>::R>& W,
                      int check_every) {
    KState* st = kstate(g, st_off);
    const long long n = g->d.n;
    OF_CUDA(cudaMemsetAsync(pa, 0, sizeof(T) * n, g->stream));
    KState h;
    if (!g->no_graphs && std::getenv("OF_NO_GRAPHS") == nullptr) {
        Graphs& G = graphs(g);
        const void* key[8] = {x, r, pa, pb, Ap, st, &W, (const void*)(uintptr_t)sizeof(T)};
        const double consts[3] = {(double)a, Q.x, Q.y};
        PlainGraph* e = nullptr;
        for (auto& c : G.plain)
            if (!std::memcmp(c.key, key, sizeof(key)) && !std::memcmp(c.consts, consts, sizeof(consts))) e = &c;
        if (!e) {
            PlainGraph c{};
            std::memcpy(c.key, key, sizeof(key));
            std::memcpy(c.consts, consts, sizeof(consts));
            c.exec = capture(g, [&] {
                krylov_step<T>(g, st, x, r, pa, pb, Ap, a, Q, W);
                krylov_step<T>(g, st, x, r, pb, pa, Ap, a, Q, W);
            }, c.kernels, c.bytes);
            G.plain.push_back(c);
            e = &G.plain.back();
        }
        const int pairs = std::max(1, check_every / 2);
        for (;;) {
            for (int k = 0; k < pairs; ++k) replay(g, e->exec, e->kernels, e->bytes, PC_KRYLOV_GRAPH);
            fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
            if (h.done != 0.0) break;
        }
        return h;
    }
    T* p[2] = {pa, pb};
    int ping = 0;
    for (;;) {
        for (int k = 0; k < check_every; ++k) {
            krylov_step<T>(g, st, x, r, p[ping], p[1 - ping], Ap, a, Q, W);
            ping ^= 1;
        }
        fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
        if (h.done != 0.0) break;
    }
    return h;
}

void destroy_graphs(void* p) { destroy_graphs_impl(p); }

__global__ void k_loop_continue(cudaGraphConditionalHandle h, const KState* st) {
    pdl_enter();
    cudaGraphSetConditional(h, st->done == 0.0 ? 1u : 0u);
}

// A launched loop graph (capture_loop) whose state has not been read back yet: its kernel
// count and algorithmic bytes follow from the iterations it ran, once the host has them.
struct PendingLoop {
    int cls = -1;
    bool sampled = false;   // the launch was timed: its profile record gets the bytes
    unsigned long long init_kernels = 0, pair_kernels = 0;
    double init_bytes = 0.0, pair_bytes = 0.0;
    void account(of_grid* g, double iters) const {
        if (cls < 0) return;
        const double pairs = std::max(1.0, std::ceil(iters / 2.0));
        __atomic_add_fetch(&g_launch_count, init_kernels + (unsigned long long)pairs * pair_kernels,
                           __ATOMIC_RELAXED);
        if (sampled && g->prof) g->prof->amend_last(cls, init_bytes + pairs * pair_bytes);
    }
};

// Launches a loop graph.  pending == nullptr: reads the solver state back (one
// synchronisation) and returns it; else returns at once (done = -1) and the caller reads the
// state later and calls pending->account.
static KState replay_loop(of_grid* g, cudaGraphExec_t exec, int st_off, int cls,
                          unsigned long long init_kernels, double init_bytes,
                          unsigned long long pair_kernels, double pair_bytes, PendingLoop* pending) {
    PendingLoop pl;
    pl.cls = cls;
    pl.init_kernels = init_kernels;
    pl.pair_kernels = pair_kernels;
    pl.init_bytes = init_bytes;
    pl.pair_bytes = pair_bytes;
    {
        ProfScope ps(g, cls, 0.0);
        OF_CUDA(cudaGraphLaunch(exec, g->stream));
        pl.sampled = ps.e0 != nullptr;
    }
    KState h{};
    if (pending) {
        *pending = pl;
        h.done = -1.0;
        return h;
    }
    fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
    pl.account(g, h.iters);
    return h;
}

// COCG on the complex shifted operator A = a(-L) + Q in FP32, preconditioned by one V-cycle of
// the real positive operator -L + sigma applied to real and imaginary parts (sigma = |Q| / a).
// Pairs of iterations replay from cached CUDA graphs as for the Poisson PCG.
static KState iterate_pcocg(of_grid* g, int st_off, float2* x, float2* r, float2* pa, float2* pb,
                            float2* Ap, float2* z, float a, double2 Q, double sigma, int check_every,
                            PendingLoop* pending = nullptr) {
    KState* st = kstate(g, st_off);
    const long long n = g->d.n;
    OF_CUDA(cudaMemsetAsync(pa, 0, sizeof(float2) * n, g->stream));
    KState h;
    if (!g->no_graphs && std::getenv("OF_NO_GRAPHS") == nullptr) {
        Graphs& G = graphs(g);
        const void* key[8] = {x, r, pa, pb, Ap, z, st, g->mg};
        const double consts[4] = {(double)a, Q.x, Q.y, sigma};
        PcocgGraph* e = nullptr;
        for (auto& c : G.pcocg)
            if (!std::memcmp(c.key, key, sizeof(key)) && !std::memcmp(c.consts, consts, sizeof(consts))) e = &c;
        if (!e) {
            PcocgGraph c{};
            std::memcpy(c.key, key, sizeof(key));
            std::memcpy(c.consts, consts, sizeof(consts));
            c.loop = capture_loop(
                g, st, [&] { pcocg_init_body(g, r, z, st, sigma); },
                [&] {
                    pcocg_step_body(g, x, r, pa, pb, Ap, z, st, a, Q, sigma);
                    pcocg_step_body(g, x, r, pb, pa, Ap, z, st, a, Q, sigma);
                },
                c.init_kernels, c.init_bytes, c.pair_kernels, c.pair_bytes);
            G.pcocg.push_back(c);
            e = &G.pcocg.back();
        }
        return replay_loop(g, e->loop, st_off, PC_PCOCG_GRAPH, e->init_kernels, e->init_bytes,
                           e->pair_kernels, e->pair_bytes, pending);
    }
    float2* p[2] = {pa, pb};
    int ping = 0;
    pcocg_init_body(g, r, z, st, sigma);
    const int every = std::max(1, check_every / 4);
    for (;;) {
        for (int k = 0; k < every; ++k) {
            pcocg_step_body(g, x, r, p[ping], p[1 - ping], Ap, z, st, a, Q, sigma);
            ping ^= 1;
        }
        fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
        if (h.done != 0.0) break;
    }
    return h;
}

// Preconditioned CG (multigrid V-cycle) on A = -L in FP32.  Without profiling the iterations
// run as replays of captured CUDA graphs; with profiling on, as individual launches so that
// every kernel class can be timed.
static KState iterate_pcg(of_grid* g, int st_off, float* x, float* r, float* pa, float* pb,
                          float* Ap, float* z, int check_every, PendingLoop* pending = nullptr) {
    KState* st = kstate(g, st_off);
    const long long n = g->d.n;
    OF_CUDA(cudaMemsetAsync(pa, 0, sizeof(float) * n, g->stream));
    KState h;
    const bool use_graphs = !g->no_graphs && std::getenv("OF_NO_GRAPHS") == nullptr;
    if (use_graphs) {
        PcgGraphs& G = graphs(g).pcg;
        const void* key[8] = {x, r, pa, pb, Ap, z, st, g->mg};
        if (!G.loop || std::memcmp(key, G.key, sizeof(key)) != 0) {
            if (G.loop) cudaGraphExecDestroy(G.loop);
            G.loop = nullptr;
            G.loop = capture_loop(
                g, st, [&] { pcg_init_body(g, r, z, st); },
                [&] {
                    pcg_step_body(g, x, r, pa, pb, Ap, z, st);
                    pcg_step_body(g, x, r, pb, pa, Ap, z, st);
                },
                G.init_kernels, G.init_bytes, G.pair_kernels, G.pair_bytes);
            std::memcpy(G.key, key, sizeof(key));
        }
        return replay_loop(g, G.loop, st_off, PC_PCG_GRAPH, G.init_kernels, G.init_bytes,
                           G.pair_kernels, G.pair_bytes, pending);
    }
    float* p[2] = {pa, pb};
    int ping = 0;
    pcg_init_body(g, r, z, st);
    const int every = std::max(1, check_every / 4);
    for (;;) {
        for (int k = 0; k < every; ++k) {
            pcg_step_body(g, x, r, p[ping], p[1 - ping], Ap, z, st);
            ping ^= 1;
        }
        fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
        if (h.done != 0.0) break;
    }
    return h;
}

// r = b - A x like OpResidual, with the Laplacian of x from its double-float split xf, summed on
// the FP32 pipes and returned to FP64 for the rest: within ~1e-13 of the FP64 sweep's value
// relative to the largest tap term, in half its time (the FP64 sweep is bound by GB300's FP64
// rate).
template <typename T64>
struct OpResidualFF {
    using TF = typename std::conditional<KT<T64>::cplx, FF2, FF>::type;
    static constexpr int kClass = KT<T64>::cplx ? PC_COCG_F64 : PC_STENCIL_F64, kWords = 3;
    const TF* xf;
    const T64* x;
    const T64* b;
    T64* r;
    KState* st;
    RedCtx rc;
    double a;
    double2 Q;
    double acc[3];
    __device__ bool begin() { acc[0] = acc[1] = acc[2] = 0.0; return true; }
    __device__ TF load(long long i) const { return xf[i]; }
    __device__ void store(long long i, TF, TF lap) {
        const T64 rv = vsub(b[i], apply_A(x[i], ff_to(lap), a, Q));
        r[i] = rv;
        acc[0] += hn2(rv);
        const double2 s = bil(rv, rv);
        acc[1] += s.x;
        acc[2] += s.y;
    }
    __device__ void end() {
        if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) &&
            threadIdx.x == 0 && threadIdx.y == 0) {
            st->rr = acc[0];
            st->rho_re = acc[1];
            st->rho_im = acc[2];
            st->beta_re = st->beta_im = 0.0;
            st->breakdown = 0.0;
            st->zshift = 0.0;
            st->done = (acc[0] <= st->tol2) ? 1.0 : 0.0;
        }
    }
};

// The double-float sweep's accuracy floor (~1e-13 of the largest tap term) sits well below the
// tolerances it serves; tighter solves keep the FP64 sweep.
constexpr double FF_MIN_TOL = 1e-11;

// ff: the Laplacian in double-float arithmetic (the mixed-precision form's refinement
// residuals); else in FP64
template <typename T>
static void residual(of_grid* g, int st_off, const T* x, const T* b, T* r, double a, double2 Q,
                     bool ff = false) {
    constexpr int RY = KT<T>::cplx ? 1 : 2;
    if (ff) {
        using TF = typename OpResidualFF<T>::TF;
        const long long n = g->d.n;
        TF* xf = (TF*)ws(g, WS_FF, sizeof(TF) * (size_t)n);
        launch(k_ff_split<T, TF>, vec_blocks(n), 256, g->stream, n, x, xf);
        OpResidualFF<T> op{xf, x, b, r, kstate(g, st_off), red_ctx(g, 0), a, Q};
        launch_stencil<TF, RY>(g, ff_weights(g->w64), op);
        return;
    }
    OpResidual<T> op{x, b, r, kstate(g, st_off), red_ctx(g, 0), (typename KT<T>::R)a, Q};
    launch_stencil<T, RY>(g, g->w64, op);
}

// Solve A x = b (b already formed in arena b64, FP64), A = a(-L) + Q.  x: FP64 guess/solution.
template <typename T64, typename T32>
static of_status solve_formed(of_grid* g, T64* x, double a, double2 Q, const KrylovOpts& o,
                              of_solve_info* info) {
    Arena ar = arena(g);
    const long long n = g->d.n;
    KState* st = kstate(g, KS64);
    T64* b = (T64*)ar.b64;
    T64* r = (T64*)ar.r64;
    launch(k_init_state, 1, 1, g->stream, st, o.max_iter);
    launch(k_norm_to_tol<T64>, vec_blocks(n), 256, g->stream, n, b, o.tol, st, red_ctx(g, 0));
    OF_LAUNCH_CHECK();
    const bool ff_res = o.precision == OF_F32 && o.tol >= FF_MIN_TOL;
    residual<T64>(g, KS64, x, b, r, a, Q, ff_res);
    KState h;
    fetch_scalars(g, KS64, KSTATE_DOUBLES, (double*)&h);
    const double bb = h.tol2 / (o.tol * o.tol);
    // a NaN or an infinity would compare false against every tolerance and pass for a zero
    // right-hand side or a converged start: refuse it instead
    OF_REQUIRE(std::isfinite(bb), OF_EINVAL, "Krylov solve: the right-hand side is not finite");
    OF_REQUIRE(std::isfinite(h.rr), OF_EINVAL,
               "Krylov solve: the initial guess gives a non-finite residual");
    int total_iters = 0, refinements = 1;
    double net_steps = 0.0;
    of_status status = OF_OK;
    if (!(bb > 0.0)) {   // zero right-hand side: the solution is zero
        OF_CUDA(cudaMemsetAsync(x, 0, sizeof(T64) * n, g->stream));
        h.rr = 0.0;
    }
    while (bb > 0.0 && h.rr > h.tol2) {
        if (total_iters >= o.max_iter || refinements > 200) { status = OF_ENOCONV; break; }
        bool residual_done = false;   // this pass read the true residual back already
        if (o.precision == OF_F32) {
            KState* s32 = kstate(g, KS32);
            T32* r32 = (T32*)ar.r32;
            T32* e32 = (T32*)ar.e32;
            // which inner solver: flexible CG with the network, multigrid-preconditioned CG /
            // COCG, or plain CG / COCG
            bool pcg = false, fcg = false;
            const double qabs = std::sqrt(Q.x * Q.x + Q.y * Q.y);
            if constexpr (std::is_same<T32, float2>::value) {
                // A shift close to the negative real axis makes a(-L) + Q nearly singular on
                // the shell of modes where a lambda = -Re Q; the V-cycle of the positive
                // operator -L + |Q| / a does not reach those modes, and each of its iterations
                // costs ~4.6x a plain one (measured on the 96^3 grid: the K_11 shift
                // -0.512 - 0.027i took 6,000-8,700 preconditioned iterations per solve), so such
                // shifts take plain COCG
                const bool near_resonant = Q.x < 0.0 && std::fabs(Q.y) < 0.2 * std::fabs(Q.x);
                // with a learned network: flexible GMRES, the network applied to the real and
                // imaginary parts of the Arnoldi vectors
                fcg = o.precond != nullptr && qabs > 0.0;
                pcg = !fcg && qabs > 0.0 && !near_resonant && !o.no_multigrid && mg_available(g);
            } else {
                const bool poisson_op = a == 1.0 && Q.x == 0.0 && Q.y == 0.0;
                fcg = poisson_op && o.precond != nullptr;
                pcg = poisson_op && !fcg && !o.no_multigrid && mg_available(g);
            }
            // A multigrid-preconditioned pass normally needs a few dozen iterations; one that
            // has not converged after MG_PASS_CAP has stalled in FP32, and the next pass
            // restarts the recurrence from the true FP64 residual.
            constexpr int MG_PASS_CAP = 100;
            const int pass_max = pcg ? std::min(MG_PASS_CAP, o.max_iter - total_iters)
                                     : o.max_iter - total_iters;
            // The pass reduces its residual by inner_tol, or by less when less is left to do: a
            // pass that started at relative residual rho only needs tol / rho, and one taken
            // further would overshoot the target (a second pass of a 1e-5 solve ran on to 1e-9).
            // The factor 0.5 leaves room for the gap between the FP32 recurrence and the true
            // residual.
            const double need = std::sqrt(h.tol2 / h.rr);   // tol / current relative residual
            const double itol = std::max(o.inner_tol, std::min(0.5, 0.5 * need));
            launch(k_demote<T64, T32>, vec_blocks(n), 256, g->stream,
                n, r, r32, e32, itol, st, s32, pass_max, red_ctx(g, 0));
            OF_LAUNCH_CHECK();
            KState hi;
            PendingLoop pending;   // a loop graph whose state is read with the outer residual
            if constexpr (std::is_same<T32, float2>::value) {
                // shifted systems: COCG preconditioned by the V-cycle of -L + |Q| / a, or
                // flexible GMRES with the network
                if (fcg)
                    hi = iterate_fgmres(g, o.precond, o.theta, KS32, e32, r32, (float*)ar.z32,
                                        (float*)ar.pb32, (float)a, Q, &net_steps);
                else if (pcg)
                    hi = iterate_pcocg(g, KS32, e32, r32, (float2*)ar.pa32, (float2*)ar.pb32,
                                       (float2*)ar.Ap32, (float2*)ar.z32, (float)a, Q, qabs / a,
                                       o.check_every, &pending);
            }
            if constexpr (std::is_same<T32, float>::value) {
                if (fcg)
                    hi = iterate_fcg(g, o.precond, o.theta, KS32, e32, r32, (float*)ar.pa32,
                                     (float*)ar.z32, o.check_every, nullptr, &net_steps, 0.0);
                else if (pcg)
                    hi = iterate_pcg(g, KS32, e32, r32, (float*)ar.pa32, (float*)ar.pb32,
                                     (float*)ar.Ap32, (float*)ar.z32, o.check_every, &pending);
            }
            if (!pcg && !fcg)
                hi = iterate<T32>(g, KS32, e32, r32, (T32*)ar.pa32, (T32*)ar.pb32,
                                  (T32*)ar.Ap32, (float)a, Q, g->w32, o.check_every);
            launch(k_promote_add<T64, T32>, vec_blocks(n), 256, g->stream, n, x, (const T32*)e32, (const KState*)s32);
            OF_LAUNCH_CHECK();
            if (hi.done == -1.0) {
                // one read-back for both states: the inner pass and the true residual after it
                // (a pass that broke down at its start has a zero correction)
                residual<T64>(g, KS64, x, b, r, a, Q, ff_res);
                static_assert(KS32 > KS64, "KState layout");
                double both[KS32 - KS64 + KSTATE_DOUBLES];
                fetch_scalars(g, KS64, KS32 - KS64 + KSTATE_DOUBLES, both);
                std::memcpy(&h, both, sizeof(KState));
                std::memcpy(&hi, both + (KS32 - KS64), sizeof(KState));
                pending.account(g, hi.iters);
                residual_done = true;
            }
            total_iters += (int)hi.iters;
            if (hi.breakdown != 0.0 && hi.iters == 0) {
                status = OF_EBREAKDOWN;
                set_error("Krylov solve (FP32 inner, %s): breakdown at the start of refinement pass "
                          "%d: inner |r|^2 %.3e, r^T M r %.3e, p^T A p %.3e, outer |r|^2 %.3e, tol2 %.3e",
                          fcg ? "flexible CG/GMRES" : pcg ? "multigrid-preconditioned CG/COCG" : "CG/COCG", refinements, hi.rr, hi.rho_re, hi.pAp_re,
                          h.rr, h.tol2);
                break;
            }
        } else {
            KState hi = iterate<T64>(g, KS64, x, r, (T64*)ar.pa64, (T64*)ar.pb64, (T64*)ar.Ap64,
                                     a, Q, g->w64, o.check_every);
            total_iters = (int)hi.iters;
            if (hi.breakdown != 0.0 && hi.rr > hi.tol2) {
                status = OF_EBREAKDOWN;
                set_error("Krylov solve (FP64): breakdown after %d iterations: |r|^2 %.3e, p^T A p %.3e",
                          total_iters, hi.rr, hi.pAp_re);
                break;
            }
        }
        if (!residual_done) {
            residual<T64>(g, KS64, x, b, r, a, Q, ff_res);   // true residual; restarts the recurrence
            fetch_scalars(g, KS64, KSTATE_DOUBLES, (double*)&h);
        }
        ++refinements;
    }
    if (info) {
        info->iterations += total_iters;
        info->refinements += refinements;
        info->rel_residual = bb > 0 ? std::sqrt(h.rr / bb) : 0.0;
        info->net_steps += (int)net_steps;
    }
    if (status == OF_ENOCONV)
        set_error("Krylov solve: %d iterations, relative residual %.3e > tol %.1e", total_iters,
                  bb > 0 ? std::sqrt(h.rr / bb) : 0.0, o.tol);
    return status;
}

static void remove_mean(of_grid* g, double* x) {
    const long long n = g->d.n;
    launch(k_sum_product, vec_blocks(n), 256, g->stream, n, x, nullptr, red_ctx(g, 120));
    launch(k_sub_mean, vec_blocks(n), 256, g->stream, n, x, g->s.scalars + 120);
    OF_LAUNCH_CHECK();
}

static of_status poisson_impl(of_grid* g, const double* a, const double* b, double* phi,
                              const KrylovOpts& o, of_solve_info* info) {
    const long long n = g->d.n;
    Arena ar = arena(g);
    launch(k_sum_product, vec_blocks(n), 256, g->stream, n, a, b, red_ctx(g, 120));
    launch(k_form_rhs, vec_blocks(n), 256, g->stream, n, a, b, g->s.scalars + 120, 4.0 * M_PI,
                                                     (double*)ar.b64);
    OF_LAUNCH_CHECK();
    of_status st = solve_formed<double, float>(g, phi, 1.0, make_double2(0.0, 0.0), o, info);
    remove_mean(g, phi);
    return st;
}

of_status poisson(of_grid* g, const double* rho, double* phi, const KrylovOpts& o,
                  of_solve_info* info) {
    return poisson_impl(g, rho, nullptr, phi, o, info);
}

of_status poisson_product(of_grid* g, const double* a, const double* b, double* phi,
                          const KrylovOpts& o, of_solve_info* info) {
    return poisson_impl(g, a, b, phi, o, info);
}

of_status shifted(of_grid* g, const double* f, double2 P, double2 Q, double kf2, double2* W,
                  const KrylovOpts& o, of_solve_info* info) {
    const long long n = g->d.n;
    Arena ar = arena(g);
    launch(k_scale_complex, vec_blocks(n), 256, g->stream, n, f, P, (double2*)ar.b64);
    OF_LAUNCH_CHECK();
    return solve_formed<double2, float2>(g, W, 1.0 / kf2, Q, o, info);
}

}  // namespace of

using namespace of;

extern "C" {

void of_default_solve_opts(of_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 20000;
    o->precision = OF_F64;
    o->inner_tol = 1e-5;
    o->check_every = 8;
    o->no_multigrid = 0;
    o->precond = nullptr;
    o->precond_theta = 0.3;
}

of_status of_poisson_solve(of_grid* g, const double* rho, double* phi, const of_solve_opts* opts,
                           of_solve_info* info) {
    if (!g || !rho || !phi) { set_error("of_poisson_solve: null argument"); return OF_EINVAL; }
    try {
        if (info) std::memset(info, 0, sizeof(*info));
        return poisson(g, rho, phi, krylov_opts(opts), info);
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_kernel_solve(of_grid* g, const double* f, int nshift, const double* P,
                          const double* Q, double kf2, double* W, const of_solve_opts* opts,
                          of_solve_info* info) {
    if (!g || !f || !P || !Q || !W || nshift < 1 || !(kf2 > 0)) {
        set_error("of_kernel_solve: bad argument");
        return OF_EINVAL;
    }
    try {
        if (info) std::memset(info, 0, sizeof(*info));
        KrylovOpts o = krylov_opts(opts);
        of_status worst = OF_OK;
        for (int s = 0; s < nshift; ++s) {
            of_solve_info one{};
            of_status st = shifted(g, f, make_double2(P[2 * s], P[2 * s + 1]),
                                   make_double2(Q[2 * s], Q[2 * s + 1]), kf2,
                                   (double2*)W + (size_t)s * g->d.n, o, &one);
            if (info) {
                info->iterations += one.iterations;
                info->refinements += one.refinements;
                info->net_steps += one.net_steps;
                info->rel_residual = std::max(info->rel_residual, one.rel_residual);
            }
            if (st != OF_OK && worst == OF_OK) worst = st;
        }
        return worst;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation Poisson solve
// A variant of the FP64 CG Poisson solve for callers that cannot call cudaMalloc (for example
// code running under an allocator it does not own, or in a process whose device memory is
// reserved up front): every buffer it needs beyond the caller's rho and phi -- the five Krylov
// vectors, the reduction partials, the block counter and the solver scalars -- lives in the
// file-scope array below.  Each GPU that loads the library holds that array until the process
// exits; all calls share it.
namespace of {

constexpr long long NOALLOC_MAX_POINTS = 1LL << 18;   // 262,144 grid points, e.g. 64^3
constexpr int NOALLOC_RED_SLOTS = 3;                  // reductions of this path use <= 3 sums
constexpr size_t NOALLOC_VEC = (size_t)NOALLOC_MAX_POINTS;
constexpr size_t NOALLOC_PARTIALS = 5 * NOALLOC_VEC;
constexpr size_t NOALLOC_SCALARS = NOALLOC_PARTIALS + (size_t)NOALLOC_RED_SLOTS * OF_MAX_RED_BLOCKS;
constexpr size_t NOALLOC_COUNTER = NOALLOC_SCALARS + 256;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_COUNTER + 8;   // about 10.6 MB

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// Device address of the scratch array, looked up once per device with that device current.
static double* noalloc_base(int device) {
    static double* addr[256] = {};
    static bool looked_up[256] = {};
    static std::mutex guard;
    OF_REQUIRE(device >= 0 && device < 256, OF_EINVAL, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(guard);
    if (!looked_up[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error("cudaGetSymbolAddress of the no-allocation scratch: %s", cudaGetErrorString(e));
            throw Error{OF_ECUDA};
        }
        addr[device] = (double*)p;
        looked_up[device] = true;
    }
    return addr[device];
}

}  // namespace of

extern "C" of_status of_poisson_solve_noalloc(int n1, int n2, int n3, double L1, double L2,
                                              double L3, int fd_half_order, void* stream,
                                              const double* rho, double* phi,
                                              const of_solve_opts* opts, of_solve_info* info) {
    using namespace of;
    if (!rho || !phi) { set_error("of_poisson_solve_noalloc: null argument"); return OF_EINVAL; }
    if (n1 < 1 || n2 < 1 || n3 < 1 || !(L1 > 0) || !(L2 > 0) || !(L3 > 0)) {
        set_error("of_poisson_solve_noalloc: bad sizes n=(%d,%d,%d) L=(%g,%g,%g)", n1, n2, n3, L1, L2, L3);
        return OF_EINVAL;
    }
    const long long n = (long long)n1 * n2 * n3;
    if (n > NOALLOC_MAX_POINTS) {
        set_error("of_poisson_solve_noalloc: %lld grid points exceed the no-allocation limit of "
                  "%lld points", n, NOALLOC_MAX_POINTS);
        return OF_EINVAL;
    }
    if (fd_half_order != 1 && fd_half_order != 3 && fd_half_order != 6) {
        set_error("of_poisson_solve_noalloc: fd_half_order %d not in {1, 3, 6}", fd_half_order);
        return OF_EINVAL;
    }
    KrylovOpts o = krylov_opts(opts);
    if (o.precision != OF_F64) {
        set_error("of_poisson_solve_noalloc: only the FP64 solve (precision OF_F64) is available");
        return OF_EINVAL;
    }
    try {
        if (info) std::memset(info, 0, sizeof(*info));
        int device = 0;
        OF_CUDA(cudaGetDevice(&device));
        double* base = noalloc_base(device);
        // A handle on the stack describing the grid; its workspace pool stays empty and
        // every pointer below points into the scratch array.
        of_grid g{};
        g.d = Dims{n1, n2, n3, n};
        g.L[0] = L1; g.L[1] = L2; g.L[2] = L3;
        const int nn[3] = {n1, n2, n3};
        for (int a = 0; a < 3; ++a) g.h[a] = g.L[a] / nn[a];
        g.dV = g.h[0] * g.h[1] * g.h[2];
        g.N = fd_half_order;
        g.w64.centre = 0.0;
        for (int a = 0; a < 3; ++a) {
            fd_weights(g.N, g.h[a], g.w64.w[a]);
            g.w64.centre += 2.0 * g.w64.w[a][0];
            for (int p = 0; p <= OF_MAX_N; ++p) g.w32.w[a][p] = (float)g.w64.w[a][p];
        }
        g.w32.centre = (float)g.w64.centre;
        g.stream = (cudaStream_t)stream;
        g.device = device;
        // no CUDA graphs: capturing one creates a capture stream and an executable graph, and
        // this handle, which never reaches of_grid_destroy, could not release them
        g.no_graphs = true;
        double host_scalars[256];
        g.s.partials = base + NOALLOC_PARTIALS;
        g.s.scalars = base + NOALLOC_SCALARS;
        g.s.counter = (unsigned int*)(base + NOALLOC_COUNTER);
        g.s.host = host_scalars;
        // the array keeps the previous call's contents: zero what must start at zero
        OF_CUDA(cudaMemsetAsync(g.s.counter, 0, sizeof(double) * 8, g.stream));
        OF_CUDA(cudaMemsetAsync(g.s.scalars, 0, sizeof(double) * 256, g.stream));

        double* r = base;
        double* pa = base + NOALLOC_VEC;
        double* pb = base + 2 * NOALLOC_VEC;
        double* Ap = base + 3 * NOALLOC_VEC;
        double* b = base + 4 * NOALLOC_VEC;
        // right-hand side 4 pi (rho - mean rho) of Eq. Poisson
        launch(k_sum_product, vec_blocks(n), 256, g.stream, n, rho, nullptr, red_ctx(&g, 120));
        launch(k_form_rhs, vec_blocks(n), 256, g.stream, n, rho, nullptr, g.s.scalars + 120,
               4.0 * M_PI, b);
        KState* st = kstate(&g, KS64);
        launch(k_init_state, 1, 1, g.stream, st, o.max_iter);
        launch(k_norm_to_tol<double>, vec_blocks(n), 256, g.stream, n, (const double*)b, o.tol, st,
               red_ctx(&g, 0));
        residual<double>(&g, KS64, phi, b, r, 1.0, make_double2(0.0, 0.0));
        KState h;
        fetch_scalars(&g, KS64, KSTATE_DOUBLES, (double*)&h);
        const double bb = h.tol2 / (o.tol * o.tol);
        OF_REQUIRE(std::isfinite(bb), OF_EINVAL,
                   "of_poisson_solve_noalloc: the right-hand side is not finite");
        OF_REQUIRE(std::isfinite(h.rr), OF_EINVAL,
                   "of_poisson_solve_noalloc: the initial guess gives a non-finite residual");
        of_status status = OF_OK;
        int iters = 0, refinements = 1;
        if (!(bb > 0.0)) {
            OF_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * n, g.stream));
            h.rr = 0.0;
        }
        while (bb > 0.0 && h.rr > h.tol2) {
            if (iters >= o.max_iter || refinements > 200) { status = OF_ENOCONV; break; }
            KState hi = iterate<double>(&g, KS64, phi, r, pa, pb, Ap, 1.0, make_double2(0.0, 0.0),
                                        g.w64, o.check_every);
            iters = (int)hi.iters;
            if (hi.breakdown != 0.0 && hi.rr > hi.tol2) { status = OF_EBREAKDOWN; break; }
            residual<double>(&g, KS64, phi, b, r, 1.0, make_double2(0.0, 0.0));
            ++refinements;
            fetch_scalars(&g, KS64, KSTATE_DOUBLES, (double*)&h);
        }
        remove_mean(&g, phi);
        OF_CUDA(cudaStreamSynchronize(g.stream));
        if (info) {
            info->iterations = iters;
            info->refinements = refinements;
            info->rel_residual = bb > 0 ? std::sqrt(h.rr / bb) : 0.0;
        }
        if (status == OF_ENOCONV)
            set_error("of_poisson_solve_noalloc: %d iterations, relative residual %.3e > tol %.1e",
                      iters, bb > 0 ? std::sqrt(h.rr / bb) : 0.0, o.tol);
        if (status == OF_EBREAKDOWN) set_error("of_poisson_solve_noalloc: breakdown");
        return status;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}
