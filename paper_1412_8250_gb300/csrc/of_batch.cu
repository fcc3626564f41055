// Batched Poisson solves over many independent cells of uneven grid sizes (each its own
// of_grid): every CG phase of all cells is one grouped launch -- each thread block finds its
// cell from a prefix table, binds that cell's fields, weights and solver state, and reduces
// into that cell's partial sums -- and the lockstep FP32 CG iterations of all cells are
// replayed from one CUDA graph.  Iterative refinement in FP64 as in the single-grid solver
// (Eq. Poisson, -(1/4pi) L_h phi = rho, mean-free).  The z extent of a stencil block is
// picked per set of grid shapes by timing the candidates once (autotuner).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <type_traits>
#include <vector>

#include "of_krylov.cuh"
#include "of_pool.cuh"

namespace of {

struct BCell {
    Dims d;
    Weights<double> w64;
    Weights<float> w32;
    int tiles_x, tiles_y, nchunks, cz;
    int sblock0;            // first block of this cell in grouped stencil launches
    int vblock0, vblocks;   // first block and block count in grouped vector launches
    double *x, *b, *r64;
    float *r32, *pa, *pb, *Ap, *e32;
    KState* s64;
    KState* s32;
    unsigned int* cnt;      // [2]: stencil-launch and vector-launch reductions
};

struct BatchShared {
    double* partials;       // [3][stride]
    int stride;
};

// per-cell two-level reduction: block partials at partials[k * stride + base + local]
template <int K>
__device__ __forceinline__ bool cell_reduce(double (&v)[K], const BatchShared& S, int base,
                                            int local, int nblocks, unsigned int* counter) {
    __shared__ double sh[32][K];
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = lane < nwarps ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            if (lane == 0) S.partials[k * S.stride + base + local] = s;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(counter, 1u) == (unsigned int)nblocks - 1u);
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = tid; b < nblocks; b += nthreads)
            s += ((volatile double*)S.partials)[k * S.stride + base + b];
        s = warp_sum(s);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += sh[w][k];
            v[k] = s;
        }
        *counter = 0u;
    }
    return true;
}

__device__ __forceinline__ int find_cell(const BCell* cells, int ncells, int block, bool vec) {
    int lo = 0, hi = ncells - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        const int start = vec ? cells[mid].vblock0 : cells[mid].sblock0;
        if (start <= block) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- grouped stencil ops
// r64 = b - A x (A = -L), |r|^2 into s64 (resets the iteration scalars)
struct GResid64 {
    const BCell* C;
    BatchShared S;
    int local, nb;
    double acc;
    __device__ bool begin() { acc = 0.0; return true; }
    __device__ double load(long long i) const { return C->x[i]; }
    __device__ void store(long long i, double, double lap) {
        const double rv = C->b[i] + lap;
        C->r64[i] = rv;
        acc += rv * rv;
    }
    __device__ void end() {
        double v[1] = {acc};
        if (cell_reduce<1>(v, S, C->sblock0, local, nb, C->cnt) && threadIdx.x == 0 && threadIdx.y == 0) {
            KState* st = C->s64;
            st->rr = v[0];
            st->done = (v[0] <= st->tol2) ? 1.0 : 0.0;
        }
    }
};

// p_out = r + beta p_in (halo included), Ap = A p_out, p^T A p and alpha into s32
struct GKrylovA32 {
    const BCell* C;
    BatchShared S;
    int local, nb, ping;
    float beta;
    const float* pin;
    float accp;
    __device__ bool begin() {
        if (C->s32->done != 0.0) return false;
        beta = (float)C->s32->beta_re;
        pin = ping ? C->pb : C->pa;
        accp = 0.f;
        return true;
    }
    __device__ float load(long long i) const { return C->r32[i] + beta * pin[i]; }
    __device__ void store(long long i, float c, float lap) {
        (ping ? C->pa : C->pb)[i] = c;
        C->Ap[i] = -lap;
        accp += c * (-lap);
    }
    __device__ void end() {
        double v[1] = {(double)accp};
        if (cell_reduce<1>(v, S, C->sblock0, local, nb, C->cnt) && threadIdx.x == 0 && threadIdx.y == 0) {
            KState* st = C->s32;
            if (!(v[0] > 0.0)) {
                st->breakdown = 1.0;
                st->done = 1.0;
            } else {
                st->alpha_re = st->rho_re / v[0];
            }
        }
    }
};

// y = L x on r32 -> Ap (autotuning probe, no reductions)
struct GLap32 {
    const BCell* C;
    BatchShared S;
    int local, nb;
    __device__ bool begin() { return true; }
    __device__ float load(long long i) const { return C->r32[i]; }
    __device__ void store(long long i, float, float lap) { C->Ap[i] = lap; }
    __device__ void end() {}
};

template <typename R> __device__ __forceinline__ const Weights<R>& cell_w(const BCell& C);
template <> __device__ __forceinline__ const Weights<double>& cell_w<double>(const BCell& C) { return C.w64; }
template <> __device__ __forceinline__ const Weights<float>& cell_w<float>(const BCell& C) { return C.w32; }

template <typename T, int N, class GOp>
__global__ void __launch_bounds__(ST_THREADS)
grouped_stencil(const BCell* cells, int ncells, BatchShared S, int ping, GOp op) {
    __shared__ int s_cell;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_cell = find_cell(cells, ncells, blockIdx.x, false);
    __syncthreads();
    const BCell* C = cells + s_cell;
    const int local = blockIdx.x - C->sblock0;
    GOp o = op;
    o.C = C;
    o.S = S;
    o.local = local;
    o.nb = C->tiles_x * C->tiles_y * C->nchunks;
    if constexpr (std::is_same<GOp, GKrylovA32>::value) o.ping = ping;
    if (!o.begin()) return;
    const int bx = local % C->tiles_x;
    const int by = (local / C->tiles_x) % C->tiles_y;
    const int bz = local / (C->tiles_x * C->tiles_y);
    stencil_tile<T, N, 2, GOp>(C->d, cell_w<T>(*C), C->cz, bx, by, bz, o);
    o.end();
}

// ---------------------------------------------------------------- grouped vector kernels
constexpr int VB_ELEMS = 1024;   // elements per block of a grouped vector launch

#define CELL_VEC_PROLOGUE                                                            \
    __shared__ int s_cell;                                                           \
    if (threadIdx.x == 0) s_cell = find_cell(cells, ncells, blockIdx.x, true);       \
    __syncthreads();                                                                 \
    const BCell* C = cells + s_cell;                                                 \
    const int local = blockIdx.x - C->vblock0;                                       \
    const long long n = C->d.n;                                                      \
    const long long i0 = (long long)local * VB_ELEMS;

// x += alpha p ; r -= alpha Ap ; |r|^2 -> beta, iteration count, done (plain CG)
__global__ void __launch_bounds__(256) gk_update32(const BCell* cells, int ncells, BatchShared S,
                                                   int ping) {
    CELL_VEC_PROLOGUE
    KState* st = C->s32;
    if (st->done != 0.0) return;
    const float al = (float)st->alpha_re;
    const float* p = ping ? C->pa : C->pb;
    float part = 0.f;
    for (long long i = i0 + threadIdx.x; i < min(n, i0 + VB_ELEMS); i += blockDim.x) {
        C->e32[i] += al * p[i];
        const float rv = C->r32[i] - al * C->Ap[i];
        C->r32[i] = rv;
        part += rv * rv;
    }
    double v[1] = {(double)part};
    if (cell_reduce<1>(v, S, C->vblock0, local, C->vblocks, C->cnt + 1) && threadIdx.x == 0) {
        const double rho_old = st->rho_re;
        st->rr = v[0];
        st->iters += 1.0;
        if (v[0] <= st->tol2 || st->iters >= st->maxit) {
            st->done = 1.0;
        } else {
            st->beta_re = v[0] / rho_old;
        }
        st->rho_re = v[0];
    }
}

// r32 = r64 / s (unit RMS), e32 = 0, fresh inner state; cells already converged skip
__global__ void __launch_bounds__(256) gk_demote(const BCell* cells, int ncells, BatchShared S,
                                                 double inner_tol, int maxit) {
    CELL_VEC_PROLOGUE
    if (C->s64->done != 0.0) {
        if (local == 0 && threadIdx.x == 0) C->s32->done = 1.0;
        return;
    }
    const double inv = C->s64->rr > 0.0 ? rsqrt(C->s64->rr / (double)n) : 1.0;
    float part = 0.f;
    for (long long i = i0 + threadIdx.x; i < min(n, i0 + VB_ELEMS); i += blockDim.x) {
        const float v = (float)(C->r64[i] * inv);
        C->r32[i] = v;
        C->e32[i] = 0.f;
        C->pa[i] = 0.f;
        part += v * v;
    }
    double v[1] = {(double)part};
    if (cell_reduce<1>(v, S, C->vblock0, local, C->vblocks, C->cnt + 1) && threadIdx.x == 0) {
        KState* st = C->s32;
        st->rr = v[0];
        st->rho_re = v[0];
        st->beta_re = 0.0;
        st->scale = 1.0 / inv;
        st->tol2 = inner_tol * inner_tol * v[0];
        st->iters = 0.0;
        st->maxit = maxit;
        st->breakdown = 0.0;
        st->done = (v[0] <= st->tol2) ? 1.0 : 0.0;
    }
}

// x64 += scale * e32 for cells that ran an inner solve
__global__ void __launch_bounds__(256) gk_promote(const BCell* cells, int ncells) {
    __shared__ int s_cell;
    if (threadIdx.x == 0) s_cell = find_cell(cells, ncells, blockIdx.x, true);
    __syncthreads();
    const BCell* C = cells + s_cell;
    if (C->s64->done != 0.0) return;
    const int local = blockIdx.x - C->vblock0;
    const long long n = C->d.n, i0 = (long long)local * VB_ELEMS;
    const double s = C->s32->scale;
    for (long long i = i0 + threadIdx.x; i < min(n, i0 + VB_ELEMS); i += blockDim.x)
        C->x[i] += s * (double)C->e32[i];
}

// |b|^2 -> s64 tol2 ; fresh outer state
__global__ void __launch_bounds__(256) gk_norm(const BCell* cells, int ncells, BatchShared S,
                                               double tol, int maxit) {
    CELL_VEC_PROLOGUE
    float part = 0.f;
    for (long long i = i0 + threadIdx.x; i < min(n, i0 + VB_ELEMS); i += blockDim.x) {
        const float v = (float)C->b[i];
        part += v * v;
    }
    double v[1] = {(double)part};
    if (cell_reduce<1>(v, S, C->vblock0, local, C->vblocks, C->cnt + 1) && threadIdx.x == 0) {
        KState* st = C->s64;
        st->tol2 = tol * tol * v[0];
        st->red[1] = v[0];
        st->iters = 0.0;
        st->maxit = maxit;
        st->done = 0.0;
        st->breakdown = 0.0;
    }
}

// ---------------------------------------------------------------- host side
struct BatchPlan {
    std::vector<BCell> h;
    BCell* d = nullptr;
    int sblocks = 0, vblocks = 0;
    BatchShared S{};
    KState* states = nullptr;
    unsigned int* counters = nullptr;
};

static void blocking(BCell& c, int cz) {
    c.tiles_x = (c.d.n1 + ST_BX - 1) / ST_BX;
    c.tiles_y = (c.d.n2 + 2 * ST_BY - 1) / (2 * ST_BY);
    c.cz = std::min(cz, c.d.n3);
    c.nchunks = (c.d.n3 + c.cz - 1) / c.cz;
}

static void layout(BatchPlan& P, int cz) {
    P.sblocks = P.vblocks = 0;
    for (auto& c : P.h) {
        blocking(c, cz);
        c.sblock0 = P.sblocks;
        P.sblocks += c.tiles_x * c.tiles_y * c.nchunks;
        c.vblock0 = P.vblocks;
        c.vblocks = (int)((c.d.n + VB_ELEMS - 1) / VB_ELEMS);
        P.vblocks += c.vblocks;
    }
}

template <class GOp>
static void grouped(of_grid* g0, BatchPlan& P, int N, int ping, GOp op, bool fp64) {
    ProfScope ps(g0, fp64 ? PC_STENCIL_F64 : PC_CG_F32, 0.0);
    if (fp64) {
        switch (N) {
            case 1: launch(grouped_stencil<double, 1, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
            case 3: launch(grouped_stencil<double, 3, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
            default: launch(grouped_stencil<double, 6, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
        }
    } else {
        switch (N) {
            case 1: launch(grouped_stencil<float, 1, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
            case 3: launch(grouped_stencil<float, 3, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
            default: launch(grouped_stencil<float, 6, GOp>, P.sblocks, dim3(ST_BX, ST_BY), g0->stream, P.d, (int)P.h.size(), P.S, ping, op); break;
        }
    }
}

static void upload(of_grid* g0, BatchPlan& P) {
    OF_CUDA(cudaMemcpyAsync(P.d, P.h.data(), sizeof(BCell) * P.h.size(), cudaMemcpyHostToDevice,
                            g0->stream));
}

// Autotuner: the z extent of a stencil block for this set of grid shapes, by timing a grouped
// FP32 sweep for each candidate (cached per shape set for the life of the process).
static int tune_cz(of_grid* g0, BatchPlan& P, int N) {
    static std::map<std::vector<long long>, int> cache;
    std::vector<long long> key;
    for (auto& c : P.h) { key.push_back(c.d.n1); key.push_back(c.d.n2); key.push_back(c.d.n3); }
    key.push_back(N);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int cand[] = {4, 8, 16, 32, 64};
    int best = 8;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    OF_CUDA(cudaEventCreate(&e0));
    OF_CUDA(cudaEventCreate(&e1));
    note_resource();
    note_resource();
    for (int cz : cand) {
        layout(P, cz);
        if (P.sblocks > P.S.stride) continue;
        upload(g0, P);
        GLap32 op{};
        grouped(g0, P, N, 0, op, false);   // warm
        OF_CUDA(cudaEventRecord(e0, g0->stream));
        for (int k = 0; k < 3; ++k) grouped(g0, P, N, 0, op, false);
        OF_CUDA(cudaEventRecord(e1, g0->stream));
        OF_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        OF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = cz; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cache[key] = best;
    return best;
}

static of_status poisson_batched(int nc, of_grid* const* gs, const double* const* rho,
                                 double* const* phi, const KrylovOpts& o, of_solve_info* infos) {
    of_grid* g0 = gs[0];
    const int N = g0->N;
    BatchPlan P;
    P.h.resize(nc);
    long long max_vec = 0;
    for (int c = 0; c < nc; ++c) {
        of_grid* g = gs[c];
        OF_REQUIRE(g && g->N == N && g->stream == g0->stream && g->device == g0->device, OF_EINVAL,
                   "batched solve: cell %d differs in order, stream or device from cell 0", c);
        OF_REQUIRE(rho[c] && phi[c], OF_EINVAL, "batched solve: null field for cell %d", c);
        Arena ar = arena(g);
        BCell& C = P.h[c];
        C.d = g->d;
        C.w64 = g->w64;
        C.w32 = g->w32;
        C.x = phi[c];
        C.b = (double*)ar.b64;
        C.r64 = (double*)ar.r64;
        C.r32 = (float*)ar.r32;
        C.pa = (float*)ar.pa32;
        C.pb = (float*)ar.pb32;
        C.Ap = (float*)ar.Ap32;
        C.e32 = (float*)ar.e32;
        // right-hand side 4 pi (rho - mean rho) in the cell's own arena
        const long long n = g->d.n;
        launch(k_sum_product, vec_blocks(n), 256, g->stream, n, rho[c], nullptr, red_ctx(g, 120));
        launch(k_form_rhs, vec_blocks(n), 256, g->stream, n, rho[c], nullptr, g->s.scalars + 120,
               4.0 * M_PI, C.b);
        max_vec = std::max(max_vec, n);
    }
    // device descriptors, states, counters and partials in cell 0's batch workspace
    long long total_sb_max = 0, total_vb = 0;
    for (auto& C : P.h) {
        BCell t = C;
        blocking(t, 4);
        total_sb_max += (long long)t.tiles_x * t.tiles_y * t.nchunks;
        total_vb += (C.d.n + VB_ELEMS - 1) / VB_ELEMS;
    }
    const int stride = (int)std::max(total_sb_max, total_vb);
    const size_t bytes = sizeof(BCell) * nc + sizeof(KState) * 2 * nc + sizeof(unsigned int) * 2 * nc +
                         sizeof(double) * 3 * (size_t)stride + 1024;
    static_assert(sizeof(BCell) % 8 == 0, "descriptor alignment");
    char* mem = (char*)ws(g0, WS_K7, bytes);
    P.d = (BCell*)mem;
    P.states = (KState*)(mem + sizeof(BCell) * nc);
    P.counters = (unsigned int*)(mem + sizeof(BCell) * nc + sizeof(KState) * 2 * nc);
    P.S.partials = (double*)(((uintptr_t)(P.counters + 2 * nc) + 255) & ~(uintptr_t)255);
    P.S.stride = stride;
    OF_CUDA(cudaMemsetAsync(P.counters, 0, sizeof(unsigned int) * 2 * nc, g0->stream));
    OF_CUDA(cudaMemsetAsync(P.states, 0, sizeof(KState) * 2 * nc, g0->stream));
    for (int c = 0; c < nc; ++c) {
        P.h[c].s64 = P.states + 2 * c;
        P.h[c].s32 = P.states + 2 * c + 1;
        P.h[c].cnt = P.counters + 2 * c;
    }
    const int cz = tune_cz(g0, P, N);
    layout(P, cz);
    upload(g0, P);
    const int ncells = nc;
    launch(gk_norm, P.vblocks, 256, g0->stream, P.d, ncells, P.S, o.tol, o.max_iter);

    // graph of two lockstep FP32 CG iterations over all cells
    cudaGraphExec_t pair = nullptr;
    unsigned long long pair_kernels = 0;
    double pair_bytes = 0.0;
    auto step = [&](int ping) {
        GKrylovA32 op{};
        grouped(g0, P, N, ping, op, false);
        ProfScope ps(g0, PC_UPDATE, 0.0);
        launch(gk_update32, P.vblocks, 256, g0->stream, P.d, ncells, P.S, ping);
    };
    const bool use_graphs = std::getenv("OF_NO_GRAPHS") == nullptr;
    if (use_graphs) pair = capture(g0, [&] { step(0); step(1); }, pair_kernels, pair_bytes);

    std::vector<KState> h64(nc), h32(nc);
    std::vector<int> iters(nc, 0), refinements(nc, 0);
    of_status status = OF_OK;
    int passes = 0;
    for (;;) {
        GResid64 rop{};
        grouped(g0, P, N, 0, rop, true);
        std::vector<KState> all(2 * nc);
        OF_CUDA(cudaMemcpyAsync(all.data(), P.states, sizeof(KState) * 2 * nc, cudaMemcpyDeviceToHost,
                                g0->stream));
        OF_CUDA(cudaStreamSynchronize(g0->stream));
        bool all_done = true, finite = true;
        for (int c = 0; c < nc; ++c) {
            h64[c] = all[2 * c];
            ++refinements[c];
            if (!(h64[c].rr <= h64[c].tol2)) all_done = false;
            if (!std::isfinite(h64[c].rr) || !std::isfinite(h64[c].tol2)) {
                if (finite)
                    set_error("batched Poisson solve: cell %d has a non-finite right-hand side or "
                              "residual", c);
                finite = false;
            }
        }
        if (!finite) { status = OF_EINVAL; break; }
        if (all_done) break;
        int max_it = 0;
        for (int c = 0; c < nc; ++c) max_it = std::max(max_it, iters[c]);
        if (max_it >= o.max_iter || ++passes > 200) { status = OF_ENOCONV; break; }
        launch(gk_demote, P.vblocks, 256, g0->stream, P.d, ncells, P.S, o.inner_tol, o.max_iter);
        for (;;) {
            if (use_graphs) {
                replay(g0, pair, pair_kernels, pair_bytes, PC_KRYLOV_GRAPH);
            } else {
                step(0);
                step(1);
            }
            OF_CUDA(cudaMemcpyAsync(all.data(), P.states, sizeof(KState) * 2 * nc,
                                    cudaMemcpyDeviceToHost, g0->stream));
            OF_CUDA(cudaStreamSynchronize(g0->stream));
            bool inner_done = true;
            for (int c = 0; c < nc; ++c)
                if (all[2 * c + 1].done == 0.0) inner_done = false;
            if (inner_done) break;
        }
        for (int c = 0; c < nc; ++c) {
            h32[c] = all[2 * c + 1];
            if (h64[c].rr > h64[c].tol2) iters[c] += (int)h32[c].iters;
        }
        launch(gk_promote, P.vblocks, 256, g0->stream, P.d, ncells);
    }
    if (pair) cudaGraphExecDestroy(pair);
    for (int c = 0; c < nc; ++c) {
        of_grid* g = gs[c];
        const long long n = g->d.n;
        launch(k_sum_product, vec_blocks(n), 256, g->stream, n, phi[c], nullptr, red_ctx(g, 120));
        launch(k_sub_mean, vec_blocks(n), 256, g->stream, n, phi[c], g->s.scalars + 120);
        if (infos) {
            const double bb = h64[c].red[1];
            infos[c].iterations = iters[c];
            infos[c].refinements = refinements[c];
            infos[c].rel_residual = bb > 0 ? std::sqrt(h64[c].rr / bb) : 0.0;
        }
    }
    OF_CUDA(cudaStreamSynchronize(g0->stream));
    if (status == OF_ENOCONV) set_error("batched Poisson solve: iteration limit reached");
    return status;
}

}  // namespace of

using namespace of;

namespace of {
// Multigrid form of the batched solve: the multigrid-preconditioned solver is host-driven per
// cell and, on cells of this size, latency bound, so the cells run on the stream pool and
// their kernels overlap on the GPU.
static of_status poisson_concurrent(int ncells, of_grid* const* grids, const double* const* rho,
                                    double* const* phi, const KrylovOpts& o, of_solve_info* infos) {
    return run_on_stream_pool(ncells, grids, [&](int c) {
        return poisson(grids[c], rho[c], phi[c], o, infos ? &infos[c] : nullptr);
    });
}
}  // namespace of

extern "C" of_status of_poisson_solve_batched(int ncells, of_grid* const* grids,
                                              const double* const* rho, double* const* phi,
                                              const of_solve_opts* opts, of_solve_info* infos) {
    if (ncells < 1 || !grids || !rho || !phi) {
        set_error("of_poisson_solve_batched: bad argument");
        return OF_EINVAL;
    }
    try {
        if (infos) std::memset(infos, 0, sizeof(of_solve_info) * ncells);
        const KrylovOpts o = krylov_opts(opts);
        if (o.precision == OF_F32 && !o.no_multigrid && o.precond == nullptr) {
            bool mg = true;
            for (int c = 0; c < ncells && mg; ++c) {
                OF_REQUIRE(grids[c] && grids[c]->stream == grids[0]->stream &&
                               grids[c]->device == grids[0]->device, OF_EINVAL,
                           "batched solve: cell %d differs in stream or device from cell 0", c);
                OF_REQUIRE(rho[c] && phi[c], OF_EINVAL, "batched solve: null field for cell %d", c);
                mg = mg_available(grids[c]);
            }
            if (mg) return poisson_concurrent(ncells, grids, rho, phi, o, infos);
        }
        return poisson_batched(ncells, grids, rho, phi, o, infos);
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}
