// Krylov-solver state and fused kernels shared by the single-grid solvers (of_krylov.cu) and
// the batched solver (of_batch.cu).
#pragma once

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "of_stencil.cuh"

namespace of {

// Device solver state, all doubles so it can be fetched with fetch_scalars.
struct KState {
    double rr;                  // 0  Hermitian |r|^2
    double tol2;                // 1  stop when rr <= tol2
    double rho_re, rho_im;      // 2  bilinear r^T r (= rr for real fields)
    double pAp_re, pAp_im;      // 4
    double alpha_re, alpha_im;  // 6
    double beta_re, beta_im;    // 8
    double done;                // 10
    double iters;               // 11
    double maxit;               // 12
    double breakdown;           // 13
    double red[4];              // 14 reduction outputs
    double zshift;              // 18 mean of the preconditioned vector (projected PCG), else 0
    double scale;               // 19 FP32 inner solve: correction = scale * FP32 solution
};
constexpr int KSTATE_DOUBLES = sizeof(KState) / sizeof(double);
constexpr int KS64 = 128;   // offsets in g->s.scalars
constexpr int KS32 = 160;
constexpr int KS_NEST = 256;   // inner solves of the flexible-GMRES preconditioner
static_assert(KS_NEST + KSTATE_DOUBLES <= OF_NSCALARS, "grid scalars");

inline KState* kstate(of_grid* g, int off) { return (KState*)(g->s.scalars + off); }

template <typename T> struct KT;
template <> struct KT<double> { static constexpr bool cplx = false; using R = double; };
template <> struct KT<float> { static constexpr bool cplx = false; using R = float; };
template <> struct KT<double2> { static constexpr bool cplx = true; using R = double; };
template <> struct KT<float2> { static constexpr bool cplx = true; using R = float; };

// Per-thread partial sums of FP32 fields are kept in FP32 (a thread sums only a few points;
// GB300's FP64 rate is 1/64 of FP32) and widened to FP64 for the block and grid reduction.
template <typename R> struct AccT { using type = double; };
template <> struct AccT<float> { using type = float; };

__device__ __forceinline__ float hn2f(float v) { return v * v; }
__device__ __forceinline__ float hn2f(float2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double hn2f(double v) { return v * v; }
__device__ __forceinline__ double hn2f(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ float2 bilf(float a, float b) { return make_float2(a * b, 0.f); }
__device__ __forceinline__ float2 bilf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 bilf(double a, double b) { return make_double2(a * b, 0.0); }
__device__ __forceinline__ double2 bilf(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// complex-or-real helpers: a scalar s (re, im) times a field value
__device__ __forceinline__ double cs_mul(double2 s, double v) { return s.x * v; }
__device__ __forceinline__ float cs_mul(double2 s, float v) { return (float)s.x * v; }
__device__ __forceinline__ double2 cs_mul(double2 s, double2 v) {
    return make_double2(s.x * v.x - s.y * v.y, s.x * v.y + s.y * v.x);
}
__device__ __forceinline__ float2 cs_mul(double2 s, float2 v) {
    const float a = (float)s.x, b = (float)s.y;
    return make_float2(a * v.x - b * v.y, a * v.y + b * v.x);
}
__device__ __forceinline__ double hn2(double v) { return v * v; }
__device__ __forceinline__ double hn2(float v) { return (double)v * v; }
__device__ __forceinline__ double hn2(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double hn2(float2 v) { return (double)v.x * v.x + (double)v.y * v.y; }
__device__ __forceinline__ double2 bil(double a, double b) { return make_double2(a * b, 0.0); }
__device__ __forceinline__ double2 bil(float a, float b) { return make_double2((double)a * b, 0.0); }
__device__ __forceinline__ double2 bil(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 bil(float2 a, float2 b) {
    return make_double2((double)a.x * b.x - (double)a.y * b.y, (double)a.x * b.y + (double)a.y * b.x);
}
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

template <typename T> __device__ __forceinline__ T one();
template <> __device__ __forceinline__ double one<double>() { return 1.0; }
template <> __device__ __forceinline__ float one<float>() { return 1.f; }
template <> __device__ __forceinline__ double2 one<double2>() { return make_double2(1.0, 0.0); }
template <> __device__ __forceinline__ float2 one<float2>() { return make_float2(1.f, 0.f); }

// Operator A v = a (-L v) + Q v
template <typename T>
__device__ __forceinline__ T apply_A(T c, T lap, typename KT<T>::R a, double2 Q) {
    return vadd(vmul(-a, lap), cs_mul(Q, c));
}

// ---------------------------------------------------------------- fused stencil ops
// r = b - A x ; reduces |r|^2 and r^T r into the state and resets the iteration scalars.
template <typename T>
struct OpResidual {
    static constexpr int kClass = KT<T>::cplx ? PC_COCG_F64 : PC_STENCIL_F64, kWords = 3;
    const T* x;
    const T* b;
    T* r;
    KState* st;
    RedCtx rc;
    typename KT<T>::R a;
    double2 Q;
    double acc[3];
    __device__ bool begin() { acc[0] = acc[1] = acc[2] = 0.0; return true; }
    __device__ T load(long long i) const { return x[i]; }
    __device__ void store(long long i, T c, T lap) {
        const T rv = vsub(b[i], apply_A(c, lap, a, Q));
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

// p_out = r + beta p_in (halo included), Ap = A p_out; reduces p^T A p and sets alpha.
template <typename T>
struct OpKrylovA {
    static constexpr int kClass = KT<T>::cplx ? (sizeof(typename KT<T>::R) == 8 ? PC_COCG_F64 : PC_COCG_F32)
                                              : (sizeof(typename KT<T>::R) == 8 ? PC_CG_F64 : PC_CG_F32);
    static constexpr int kWords = 4;   // read r (or z) and p, write p and A p
    const T* r;
    const T* pin;
    T* pout;
    T* Ap;
    KState* st;
    RedCtx rc;
    typename KT<T>::R a;
    double2 Q;
    double2 beta;
    double2 shift;
    typename AccT<typename KT<T>::R>::type accp[2];
    __device__ bool begin() {
        if (st->done != 0.0) return false;
        beta = make_double2(st->beta_re, st->beta_im);
        shift = make_double2(-st->zshift, 0.0);
        accp[0] = accp[1] = 0;
        return true;
    }
    // p = (r - zshift) + beta p_in ; zshift is 0 except in the projected PCG
    __device__ T load(long long i) const {
        return vadd(vadd(r[i], cs_mul(shift, one<T>())), cs_mul(beta, pin[i]));
    }
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ float2 load2(long long i) const {
        const float2 rv = *reinterpret_cast<const float2*>(r + i);
        const float2 pv = *reinterpret_cast<const float2*>(pin + i);
        const float s = (float)shift.x, b = (float)beta.x;
        return make_float2(fmaf(b, pv.x, rv.x + s), fmaf(b, pv.y, rv.y + s));
    }
    __device__ void store(long long i, T c, T lap) {
        pout[i] = c;
        const T av = apply_A(c, lap, a, Q);
        Ap[i] = av;
        const auto s = bilf(c, av);
        accp[0] += s.x;
        accp[1] += s.y;
    }
    // points i, i + 1 of a real field (i even): the same as two store calls
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ void store2(long long i, float2 c, float2 lap) {
        *reinterpret_cast<float2*>(pout + i) = c;
        const float a0 = apply_A(c.x, lap.x, a, Q), a1 = apply_A(c.y, lap.y, a, Q);
        *reinterpret_cast<float2*>(Ap + i) = make_float2(a0, a1);
        const auto s0 = bilf(c.x, a0), s1 = bilf(c.y, a1);
        accp[0] += s0.x;
        accp[1] += s0.y;
        accp[0] += s1.x;
        accp[1] += s1.y;
    }
    __device__ void end() {
        double acc[2] = {(double)accp[0], (double)accp[1]};
        if (grid_reduce<2>(acc, rc.partials, rc.counter, st->red) &&
            threadIdx.x == 0 && threadIdx.y == 0) {
            const double2 pAp = make_double2(acc[0], acc[1]);
            st->pAp_re = pAp.x;
            st->pAp_im = pAp.y;
            const double mag = fabs(pAp.x) + fabs(pAp.y);
            const bool bad = KT<T>::cplx ? !(mag > 0.0) : !(pAp.x > 0.0);
            if (bad) {
                st->breakdown = 1.0;
                st->done = 1.0;
            } else {
                const double2 al = cdiv(make_double2(st->rho_re, st->rho_im), pAp);
                st->alpha_re = al.x;
                st->alpha_im = al.y;
            }
        }
    }
};

// The scalars of a Krylov update from its grid-reduced sums acc = (|r|^2, r^T r): iteration
// count, convergence, beta (plain CG / COCG; the preconditioned forms take beta from r^T z).
template <bool PRECOND>
__device__ __forceinline__ void krylov_update_finish(const double (&acc)[3], KState* st) {
    const double2 rho_new = make_double2(acc[1], acc[2]);
    const double2 rho_old = make_double2(st->rho_re, st->rho_im);
    st->rr = acc[0];
    st->iters += 1.0;
    if (acc[0] <= st->tol2 || st->iters >= st->maxit) {
        st->done = 1.0;
    } else if (PRECOND) {
        return;   // beta follows from r^T z once the preconditioner has run
    } else if (!(fabs(rho_old.x) + fabs(rho_old.y) > 0.0)) {
        st->breakdown = 1.0;
        st->done = 1.0;
    } else {
        const double2 be = cdiv(rho_new, rho_old);
        st->beta_re = be.x;
        st->beta_im = be.y;
    }
    st->rho_re = rho_new.x;
    st->rho_im = rho_new.y;
}

// x += alpha p ; r -= alpha Ap ; reduces |r|^2 and r^T r ; sets beta, iteration count, done.
template <typename T, bool PRECOND = false>
__global__ void __launch_bounds__(256) krylov_update(long long n, T* __restrict__ x,
                                                     T* __restrict__ r, const T* __restrict__ p,
                                                     const T* __restrict__ Ap, KState* st,
                                                     RedCtx rc) {
    pdl_enter();
    if (st->done != 0.0) return;
    const double2 al = make_double2(st->alpha_re, st->alpha_im);
    typename AccT<typename KT<T>::R>::type a0 = 0, a1 = 0, a2 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] = vadd(x[i], cs_mul(al, p[i]));
        const T rv = vsub(r[i], cs_mul(al, Ap[i]));
        r[i] = rv;
        a0 += hn2f(rv);
        if (!PRECOND) {
            const auto s = bilf(rv, rv);
            a1 += s.x;
            a2 += s.y;
        }
    }
    double acc[3] = {(double)a0, (double)a1, (double)a2};
    if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0)
        krylov_update_finish<PRECOND>(acc, st);
}

// The same for FP32 fields (real, or complex as float2) moved as 16-byte vectors: nv = the
// number of float4 (n * sizeof(T) / 16), all four arrays 16-byte aligned.
template <typename T, bool PRECOND = false>
__global__ void __launch_bounds__(256) krylov_update_v4(long long nv, float4* __restrict__ x,
                                                        float4* __restrict__ r,
                                                        const float4* __restrict__ p,
                                                        const float4* __restrict__ Ap, KState* st,
                                                        RedCtx rc) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "FP32 fields only");
    constexpr int K = 16 / sizeof(T);
    pdl_enter();
    if (st->done != 0.0) return;
    const double2 al = make_double2(st->alpha_re, st->alpha_im);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        float4 xv = x[v], rv4 = r[v];
        const float4 pv = p[v], av = Ap[v];
        T* xe = reinterpret_cast<T*>(&xv);
        T* re = reinterpret_cast<T*>(&rv4);
        const T* pe = reinterpret_cast<const T*>(&pv);
        const T* ae = reinterpret_cast<const T*>(&av);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            xe[k] = vadd(xe[k], cs_mul(al, pe[k]));
            const T rk = vsub(re[k], cs_mul(al, ae[k]));
            re[k] = rk;
            a0 += hn2f(rk);
            if (!PRECOND) {
                const auto s = bilf(rk, rk);
                a1 += s.x;
                a2 += s.y;
            }
        }
        x[v] = xv;
        r[v] = rv4;
    }
    double acc[3] = {(double)a0, (double)a1, (double)a2};
    if (grid_reduce<3>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0)
        krylov_update_finish<PRECOND>(acc, st);
}

// Launches the Krylov update, as 16-byte vectors where the FP32 fields allow it.
template <typename T, bool PRECOND>
inline void launch_krylov_update(of_grid* g, long long n, T* x, T* r, const T* p, const T* Ap,
                                 KState* st, RedCtx rc, int blocks) {
    if constexpr (sizeof(typename KT<T>::R) == 4) {
        const bool aligned = (((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)Ap) & 15) == 0;
        if (aligned && (n * (long long)sizeof(T)) % 16 == 0) {
            launch_pdl(krylov_update_v4<T, PRECOND>, blocks, 256, 0, g->stream, n * (long long)sizeof(T) / 16,
                   (float4*)x, (float4*)r, (const float4*)p, (const float4*)Ap, st, rc);
            return;
        }
    }
    launch_pdl(krylov_update<T, PRECOND>, blocks, 256, 0, g->stream, n, x, r, p, Ap, st, rc);
}

inline int vec_blocks(long long n) { return red_blocks(n, 256 * 4); }

// Preconditioned-CG scalars from the grid-reduced sums s = (r^T z, sum z, sum r) (projected:
// z is used with its mean removed): rho = r^T (z - zbar), beta = rho / rho_old (0 first).
__device__ __forceinline__ void pcg_finish(KState* st, const double (&s)[3], long long n, bool first) {
    const double zbar = s[1] / (double)n;
    const double rho = s[0] - zbar * s[2];
    if (!(rho > 0.0)) {   // M^{-1} must be positive definite on r
        st->breakdown = 1.0;
        st->done = 1.0;
        return;
    }
    st->beta_re = first ? 0.0 : rho / st->rho_re;
    st->beta_im = 0.0;
    st->rho_re = rho;
    st->rho_im = 0.0;
    st->zshift = zbar;
}
// Preconditioned COCG: rho = r^T z (bilinear, complex), beta = rho / rho_old (0 first).
__device__ __forceinline__ void pcocg_finish(KState* st, const double (&s)[2], bool first) {
    const double2 rho = make_double2(s[0], s[1]);
    if (!(fabs(rho.x) + fabs(rho.y) > 0.0)) {
        st->breakdown = 1.0;
        st->done = 1.0;
        return;
    }
    const double2 beta = first ? make_double2(0.0, 0.0) : cdiv(rho, make_double2(st->rho_re, st->rho_im));
    st->beta_re = beta.x;
    st->beta_im = beta.y;
    st->rho_re = rho.x;
    st->rho_im = rho.y;
    st->zshift = 0.0;
}

// One V-cycle z = M^{-1} r (of_mg.cu) whose last smoothing sweep also forms the
// preconditioned-CG scalars (pcg_finish / pcocg_finish) on state st.  Returns false when the
// hierarchy has no grid-wide level to fuse into; the caller then reduces separately.
bool mg_vcycle_beta(of_grid* g, const float* r, float* z, KState* st, bool first);
bool mg_vcycle_shifted_beta(of_grid* g, const float2* r, float2* z, KState* st, bool first,
                            double sigma);


// Arena of Krylov vectors: FP64 (r, pa, pb, Ap, b) and FP32 (r, pa, pb, Ap, e), complex-sized.
struct Arena {
    void* r64; void* pa64; void* pb64; void* Ap64; void* b64;
    void* r32; void* pa32; void* pb32; void* Ap32; void* e32; void* z32;
};

inline Arena arena(of_grid* g) {
    const size_t n = (size_t)g->d.n;
    const size_t s64 = ((n * sizeof(double2) + 255) / 256) * 256;
    const size_t s32 = ((n * sizeof(float2) + 255) / 256) * 256;
    char* base = (char*)ws(g, WS_K0, 5 * s64 + 6 * s32);
    Arena a;
    a.r64 = base; a.pa64 = base + s64; a.pb64 = base + 2 * s64; a.Ap64 = base + 3 * s64;
    a.b64 = base + 4 * s64;
    char* b32 = base + 5 * s64;
    a.r32 = b32; a.pa32 = b32 + s32; a.pb32 = b32 + 2 * s32; a.Ap32 = b32 + 3 * s32;
    a.e32 = b32 + 4 * s32;
    a.z32 = b32 + 5 * s32;
    return a;
}


// Flexible CG with the learned preconditioner (of_precond.cu) on -L_h + shift; P == nullptr:
// plain CG.
struct Sink;
KState iterate_fcg(of_grid* g, of_precond* P, double theta, int st_off, float* x, float* r,
                   float* ra, float* z, int check_every, Sink* sink, double* net_steps,
                   double shift);
// Flexible GMRES(8) on the shifted system a (-L_h) x + Q x = b, preconditioned by flexible CG
// with the learned network on the real positive operator -L_h + |Q| / a, applied to the real
// and imaginary parts (x = 0 on entry; the KState at st_off holds |b|^2, tol2 and maxit and is
// read, not written).  x, b: n complex; z, rs: 2n floats of scratch.  Returns the outer plus
// inner iterations and the final |b - A x|^2 in rr.
KState iterate_fgmres(of_grid* g, of_precond* P, double theta, int st_off, float2* x, const float2* b,
                      float* z, float* rs, float a, double2 Q, double* net_steps);

// CUDA graphs of the preconditioned CG: "init" (V-cycle + first r^T z) and "pair" (two full
// iterations, ping and pong of the direction buffers).  Every kernel reads its scalars and the
// stop flag from device memory, so the same executable graph serves every solve on the grid's
// arena; it is rebuilt only if a buffer address changes.
struct PcgGraphs {
    const void* key[8] = {};
    cudaGraphExec_t init = nullptr, pair = nullptr;
    unsigned long long init_kernels = 0, pair_kernels = 0;
    double init_bytes = 0.0, pair_bytes = 0.0;
    cudaGraphExec_t loop = nullptr;   // init, then pair while not done (device-side loop)
};

// Graphs of two plain CG / COCG iterations, keyed by buffers and operator constants.
struct PlainGraph {
    const void* key[8];
    double consts[3];
    cudaGraphExec_t exec;
    unsigned long long kernels;
    double bytes;
};

// Graphs of the multigrid-preconditioned COCG (init + pair), keyed by buffers and constants.
struct PcocgGraph {
    const void* key[8];
    double consts[4];   // a, Q (re, im), sigma
    cudaGraphExec_t init, pair;
    unsigned long long init_kernels, pair_kernels;
    double init_bytes, pair_bytes;
    cudaGraphExec_t loop;   // init, then pair while not done (device-side loop)
};

struct Graphs {
    PcgGraphs pcg;
    std::vector<PlainGraph> plain;
    std::vector<PcocgGraph> pcocg;
};

inline void destroy_graphs_impl(void* p) {
    Graphs* G = (Graphs*)p;
    if (!G) return;
    if (G->pcg.init) cudaGraphExecDestroy(G->pcg.init);
    if (G->pcg.pair) cudaGraphExecDestroy(G->pcg.pair);
    if (G->pcg.loop) cudaGraphExecDestroy(G->pcg.loop);
    for (auto& e : G->plain)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    for (auto& e : G->pcocg) {
        if (e.init) cudaGraphExecDestroy(e.init);
        if (e.pair) cudaGraphExecDestroy(e.pair);
        if (e.loop) cudaGraphExecDestroy(e.loop);
    }
    delete G;
}

inline Graphs& graphs(of_grid* g) {
    if (!g->graphs) g->graphs = new Graphs();
    return *(Graphs*)g->graphs;
}

template <class Body>
inline cudaGraphExec_t capture(of_grid* g, Body&& body, unsigned long long& kernels,
                               double& bytes) {
    if (!g->cap_stream) {
        OF_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        note_resource();
    }
    cudaStream_t saved = g->stream;
    Prof* saved_prof = g->prof;
    g->stream = g->cap_stream;
    g->prof = nullptr;
    const unsigned long long c0 = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED);
    cudaGraph_t graph = nullptr;
    OF_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    g_capture_bytes = 0.0;
    try {
        body();
    } catch (...) {
        g_capturing = false;
        cudaStreamEndCapture(g->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        g->stream = saved;
        g->prof = saved_prof;
        throw;
    }
    g_capturing = false;
    bytes = g_capture_bytes;
    cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    g->stream = saved;
    g->prof = saved_prof;
    OF_CUDA(e);
    kernels = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED) - c0;
    __atomic_sub_fetch(&g_launch_count, kernels, __ATOMIC_RELAXED);   // captured, not launched
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    OF_CUDA(e);
    note_resource();
    return exec;
}

// Sets the condition of the enclosing WHILE node: repeat while the solver state is not done.
__global__ void k_loop_continue(cudaGraphConditionalHandle h, const KState* st);

// One executable graph for a whole preconditioned pass: `init` once, then `pair` (two
// iterations) under a conditional WHILE node whose body ends with k_loop_continue, so that the
// iterations repeat on the device until the state's done flag is set (convergence, breakdown or
// the iteration cap, all set by the kernels).  One host launch and one host synchronisation per
// pass instead of one per pair.
template <class Init, class Pair>
inline cudaGraphExec_t capture_loop(of_grid* g, KState* st, Init&& init, Pair&& pair,
                                    unsigned long long& init_kernels, double& init_bytes,
                                    unsigned long long& pair_kernels, double& pair_bytes) {
    if (!g->cap_stream) {
        OF_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        note_resource();
    }
    if (!g->cap_stream2) {
        OF_CUDA(cudaStreamCreateWithFlags(&g->cap_stream2, cudaStreamNonBlocking));
        note_resource();
    }
    cudaStream_t saved = g->stream;
    Prof* saved_prof = g->prof;
    g->prof = nullptr;
    cudaGraph_t graph = nullptr;
    bool main_open = false, body_open = false;
    auto restore = [&]() {
        g_capturing = false;
        g->stream = saved;
        g->prof = saved_prof;
    };
    try {
        unsigned long long c0 = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED);
        g->stream = g->cap_stream;
        OF_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        main_open = true;
        g_capturing = true;
        g_capture_bytes = 0.0;
        init();
        init_bytes = g_capture_bytes;
        init_kernels = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED) - c0;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        OF_CUDA(cudaStreamGetCaptureInfo(g->cap_stream, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
        cudaGraphConditionalHandle handle;
        OF_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        OF_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        c0 = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED);
        g->stream = g->cap_stream2;
        OF_CUDA(cudaStreamBeginCaptureToGraph(g->stream, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        body_open = true;
        g_capture_bytes = 0.0;
        pair();
        launch_pdl(k_loop_continue, 1, 1, 0, g->stream, handle, (const KState*)st);
        pair_bytes = g_capture_bytes;
        pair_kernels = __atomic_load_n(&g_launch_count, __ATOMIC_RELAXED) - c0;
        body_open = false;
        OF_CUDA(cudaStreamEndCapture(g->stream, nullptr));
        g->stream = g->cap_stream;
        OF_CUDA(cudaStreamUpdateCaptureDependencies(g->stream, &node, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
        main_open = false;
        OF_CUDA(cudaStreamEndCapture(g->stream, &graph));
    } catch (...) {
        if (body_open) cudaStreamEndCapture(g->cap_stream2, nullptr);
        if (main_open) {
            cudaGraph_t partial = nullptr;
            cudaStreamEndCapture(g->cap_stream, &partial);
            if (partial) cudaGraphDestroy(partial);
        }
        restore();
        throw;
    }
    restore();
    // captured, not launched
    __atomic_sub_fetch(&g_launch_count, init_kernels + pair_kernels, __ATOMIC_RELAXED);
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    OF_CUDA(e);
    note_resource();
    return exec;
}

inline void replay(of_grid* g, cudaGraphExec_t exec, unsigned long long kernels, double bytes,
                   int cls = PC_PCG_GRAPH) {
    ProfScope ps(g, cls, bytes);
    OF_CUDA(cudaGraphLaunch(exec, g->stream));
    __atomic_add_fetch(&g_launch_count, kernels, __ATOMIC_RELAXED);
}


// kernels and helpers of of_krylov.cu used by other units
__global__ void k_form_rhs(long long n, const double* a, const double* b, const double* sum_dev,
                           double scale, double* y);
__global__ void k_sub_mean(long long n, double* x, const double* sum_dev);
KrylovOpts krylov_opts(const of_solve_opts* o);

}  // namespace of
