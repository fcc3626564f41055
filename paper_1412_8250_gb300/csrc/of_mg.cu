// Geometric multigrid V-cycle used as the preconditioner of the FP32 inner CG of the Poisson
// solve.  The paper (Sec. 5.5) names multigrid as the way to stop the Poisson iteration count
// from growing with system size; this is that preconditioner on the periodic grid.
//
//  level 0   : the order-2N operator A = -L_h of Eq. FD:Laplacian (FP32)
//  level l>0 : the second-order 7-point operator at spacing 2^l h
//  transfer  : full weighting R = (1/8) P^T, trilinear prolongation P (periodic wrap)
//  smoother  : Chebyshev polynomial of the Jacobi-scaled operator on [0.15, 1.05] lambda_max,
//              degree 2 before and after the coarse correction (same polynomial both sides,
//              so the V-cycle is symmetric and fixed: a valid CG preconditioner)
//  coarsest  : Chebyshev over the whole non-zero spectrum, one thread block, when the grid
//              cannot be halved further (an odd or small dimension)
// Every kernel reads the solver's stop flag and returns at once after convergence.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "of_krylov.cuh"

namespace cg = cooperative_groups;

namespace of {

struct MGLevel {
    Dims d;
    double h[3];
    int N;
    Weights<float> W;
    double diag;             // diagonal of -L_h on this level
    double lmax, lmin;       // largest and smallest non-zero eigenvalue of -L_h
    float *x, *b, *r, *d0, *d1;   // each sized for complex (float2) fields
};

// Level parameters for the operator A = -L_h + sigma (sigma >= 0): Jacobi scaling and the
// extreme eigenvalues of D^{-1} A (the constant mode has eigenvalue sigma).
struct Shifted {
    float invD;
    double lmax, lmin;
};
static Shifted shifted_level(const MGLevel& L, double sigma) {
    const double D = L.diag + sigma;
    Shifted s;
    s.invD = (float)(1.0 / D);
    s.lmax = (L.lmax + sigma) / D;
    s.lmin = (sigma > 0.0 ? std::min(sigma, L.lmin + sigma) : L.lmin) / D;
    return s;
}

struct MG {
    std::vector<MGLevel> lv;
    int deg = 2;
    int first_small = 1;   // levels from here down run inside one thread-block cluster
    bool ok = false;
};

constexpr long long MG_SMALL_POINTS = 16384;   // levels this small run in one block
constexpr int MG_MAX_LEVELS = 10;

void mg_destroy(MG* m) { delete m; }

static void weights_for(int N, const double h[3], Weights<float>& W, double& diag) {
    double w[3][OF_MAX_N + 1];
    W.centre = 0.f;
    double c = 0.0;
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int q = 1; q <= N; ++q) s += 1.0 / ((double)q * q);
        w[a][0] = -s / (h[a] * h[a]);
        for (int p = 1; p <= N; ++p) {
            double ratio = 1.0;
            for (int k = 1; k <= p; ++k) ratio *= (double)(N - p + k) / (double)(N + k);
            w[a][p] = 2.0 * ((p % 2) ? 1.0 : -1.0) * ratio / (h[a] * h[a] * p * p);
        }
        for (int p = N + 1; p <= OF_MAX_N; ++p) w[a][p] = 0.0;
        for (int p = 0; p <= OF_MAX_N; ++p) W.w[a][p] = (float)w[a][p];
        c += 2.0 * w[a][0];
    }
    W.centre = (float)c;
    diag = -c;   // diagonal of A = -L
}

// extreme eigenvalues of D^{-1} A on the periodic grid, from the stencil's symbol per axis
static void spectrum(int N, const double h[3], const Dims& d, double diag, double& lmax,
                     double& lmin_nz) {
    lmax = 0.0;
    double smallest_axis = 1e300;
    for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? d.n1 : (a == 1 ? d.n2 : d.n3);
        double s = 0.0;
        for (int q = 1; q <= N; ++q) s += 1.0 / ((double)q * q);
        double best = 0.0, small = 1e300;
        for (int m = 0; m < n; ++m) {
            const double th = 2.0 * M_PI * m / n;
            double v = 2.0 * s;
            for (int p = 1; p <= N; ++p) {
                double ratio = 1.0;
                for (int k = 1; k <= p; ++k) ratio *= (double)(N - p + k) / (double)(N + k);
                v -= 2.0 * 2.0 * ((p % 2) ? 1.0 : -1.0) * ratio / (p * p) * std::cos(p * th);
            }
            v /= h[a] * h[a];
            best = std::max(best, v);
            if (m > 0) small = std::min(small, v);
        }
        lmax += best;
        smallest_axis = std::min(smallest_axis, small);
    }
    lmax /= diag;
    lmin_nz = smallest_axis / diag;
}

static bool build(of_grid* g, MG& m) {
    Dims d = g->d;
    double h[3] = {g->h[0], g->h[1], g->h[2]};
    int N = g->N;
    std::vector<MGLevel> lv;
    size_t total = 0;
    for (;;) {
        MGLevel L{};
        L.d = d;
        for (int a = 0; a < 3; ++a) L.h[a] = h[a];
        L.N = N;
        double diag, lmax, lmin;
        weights_for(N, h, L.W, diag);
        spectrum(N, h, d, diag, lmax, lmin);
        L.diag = diag;
        L.lmax = lmax * diag;
        L.lmin = lmin * diag;
        lv.push_back(L);
        total += 5 * (2 * (size_t)d.n + 64);
        const bool can = d.n1 % 2 == 0 && d.n2 % 2 == 0 && d.n3 % 2 == 0 && d.n1 >= 8 &&
                         d.n2 >= 8 && d.n3 >= 8;
        if (!can) break;
        d = Dims{d.n1 / 2, d.n2 / 2, d.n3 / 2, (long long)(d.n1 / 2) * (d.n2 / 2) * (d.n3 / 2)};
        for (int a = 0; a < 3; ++a) h[a] *= 2.0;
        N = 1;
    }
    if (lv.size() < 2 || lv.size() > (size_t)MG_MAX_LEVELS || lv.back().d.n > MG_SMALL_POINTS)
        return false;
    float* base = (float*)ws(g, WS_MG, sizeof(float) * (total + 64 * lv.size()));
    size_t off = 0;
    for (auto& L : lv) {
        float** p[5] = {&L.x, &L.b, &L.r, &L.d0, &L.d1};
        for (int k = 0; k < 5; ++k) {
            *p[k] = base + off;
            off += (2 * (size_t)L.d.n + 63) / 64 * 64;
        }
    }
    m.lv = lv;
    m.ok = true;
    m.first_small = (int)m.lv.size() - 1;
    while (m.first_small > 1 && m.lv[m.first_small - 1].d.n <= MG_SMALL_POINTS) --m.first_small;
    return true;
}

bool mg_available(of_grid* g) {
    if (!g->mg) {
        g->mg = new MG();
        if (!build(g, *g->mg)) g->mg->ok = false;
    }
    return g->mg->ok;
}

// ---------------------------------------------------------------- kernels
// T = float (real fields) or float2 (complex fields, real and imaginary parts smoothed alike:
// the operator is real).  A = -L_h + sigma.
// One Chebyshev step: x (+)= d ; r_out = r_in - A d ; d_out = a d + bD r_out
template <typename T>
struct OpCheby {
    static constexpr int kClass = PC_MG_SMOOTH, kWords = 6;
    const T* din;
    float dscale;
    T* x;
    bool x_init;
    const T* rin;
    T* rout;
    T* dout;
    float a, bD, sigma;
    const double* done;
    // last sweep of a V-cycle inside preconditioned CG / COCG (rk non-null): also reduce
    // r^T z, sum z, sum r (real) or the complex r^T z, z = the updated x, and finish beta
    const T* rk = nullptr;
    KState* st = nullptr;
    RedCtx rc{};
    bool first = false;
    long long n = 0;
    float acc[3];
    __device__ bool begin() {
        acc[0] = acc[1] = acc[2] = 0.f;
        return *done == 0.0;
    }
    __device__ T load(long long i) const { return vmul(dscale, din[i]); }
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ float2 load2(long long i) const {
        const float2 v = *reinterpret_cast<const float2*>(din + i);
        return make_float2(dscale * v.x, dscale * v.y);
    }
    __device__ void store(long long i, T c, T lap) {
        const T xn = x_init ? c : vadd(x[i], c);
        x[i] = xn;
        const T rn = vfma(-sigma, c, vadd(rin[i], lap));   // r - A d
        rout[i] = rn;
        if (dout) dout[i] = vfma(a, c, vmul(bD, rn));
        if (rk) accumulate(rk[i], xn);
    }
    // points i, i + 1 of a real field (i even): the same as two store calls
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ void store2(long long i, float2 c, float2 lap) {
        float2 xn = c;
        if (!x_init) {
            const float2 xo = *reinterpret_cast<const float2*>(x + i);
            xn = make_float2(xo.x + c.x, xo.y + c.y);
        }
        *reinterpret_cast<float2*>(x + i) = xn;
        const float2 ri = *reinterpret_cast<const float2*>(rin + i);
        const float2 rn = make_float2(fmaf(-sigma, c.x, ri.x + lap.x), fmaf(-sigma, c.y, ri.y + lap.y));
        *reinterpret_cast<float2*>(rout + i) = rn;
        if (dout)
            *reinterpret_cast<float2*>(dout + i) =
                make_float2(fmaf(a, c.x, bD * rn.x), fmaf(a, c.y, bD * rn.y));
        if (rk) {
            const float2 rr = *reinterpret_cast<const float2*>(rk + i);
            accumulate(rr.x, xn.x);
            accumulate(rr.y, xn.y);
        }
    }
    __device__ void accumulate(float r, float z) {
        acc[0] = fmaf(r, z, acc[0]);
        acc[1] += z;
        acc[2] += r;
    }
    __device__ void accumulate(float2 r, float2 z) {
        acc[0] = fmaf(r.x, z.x, fmaf(-r.y, z.y, acc[0]));
        acc[1] = fmaf(r.x, z.y, fmaf(r.y, z.x, acc[1]));
    }
    __device__ void end() {
        if (!rk) return;
        if constexpr (std::is_same<T, float>::value) {
            double s[3] = {(double)acc[0], (double)acc[1], (double)acc[2]};
            if (grid_reduce<3>(s, rc.partials, rc.counter, st->red) && threadIdx.x == 0 && threadIdx.y == 0)
                pcg_finish(st, s, n, first);
        } else {
            double s[2] = {(double)acc[0], (double)acc[1]};
            if (grid_reduce<2>(s, rc.partials, rc.counter, st->red) && threadIdx.x == 0 && threadIdx.y == 0)
                pcocg_finish(st, s, first);
        }
    }
};

// the CG scalars fused into a V-cycle's last sweep: (KState, first call, residual)
template <typename T>
struct BetaFuse {
    KState* st;
    bool first;
    const T* r;
};

// r = b - A x, and (d0 non-null) the first Chebyshev direction d0 = s0 r beside it: the first
// smoothing step then reads d0 at the neighbours while it rewrites r at its own points (it
// must not read r there: other blocks update r while a block stages its halo)
template <typename T>
struct OpResid32 {
    static constexpr int kClass = PC_MG_SMOOTH, kWords = 3;
    const T* x;
    const T* b;
    T* r;
    float sigma;
    const double* done;
    T* d0 = nullptr;
    float s0 = 0.f;
    __device__ bool begin() { return *done == 0.0; }
    __device__ T load(long long i) const { return x[i]; }
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ float2 load2(long long i) const { return *reinterpret_cast<const float2*>(x + i); }
    __device__ void store(long long i, T c, T lap) {
        const T rv = vfma(-sigma, c, vadd(b[i], lap));
        r[i] = rv;
        if (d0) d0[i] = vmul(s0, rv);
    }
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ void store2(long long i, float2 c, float2 lap) {
        const float2 bv = *reinterpret_cast<const float2*>(b + i);
        const float2 rv = make_float2(fmaf(-sigma, c.x, bv.x + lap.x), fmaf(-sigma, c.y, bv.y + lap.y));
        *reinterpret_cast<float2*>(r + i) = rv;
        if (d0) *reinterpret_cast<float2*>(d0 + i) = make_float2(s0 * rv.x, s0 * rv.y);
    }
    __device__ void end() {}
};

__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
template <typename T> __device__ __forceinline__ T vzero();
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }

// grid of 32 x 8 thread blocks over the points of a level, one block row per plane
static inline dim3 grid3(const Dims& d) {
    return dim3((unsigned)((d.n1 + 31) / 32), (unsigned)((d.n2 + 7) / 8), (unsigned)d.n3);
}

// coarse b = full weighting of fine r
template <typename T>
__global__ void k_restrict(Dims f, Dims c, const T* __restrict__ r, T* __restrict__ b,
                           const double* done) {
    pdl_enter();
    if (*done != 0.0) return;
    // 3-D launch (x_blocks, y_blocks, c.n3) of 32 x 8 threads: no index division
    const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
    if (I >= c.n1 || J >= c.n2) return;
    const long long idx = ((long long)K * c.n2 + J) * c.n1 + I;
    T s = vzero<T>();
    const float w[3] = {0.25f, 0.5f, 0.25f};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = wrapc(2 * K + dz, f.n3);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = wrapc(2 * J + dy, f.n2);
            const long long row = ((long long)z * f.n2 + y) * f.n1;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = wrapc(2 * I + dx, f.n1);
                s = vfma(w[dz + 1] * w[dy + 1] * w[dx + 1], r[row + x], s);
            }
        }
    }
    b[idx] = s;
}

// trilinear interpolation of the coarse field e at fine point (i, j, k)
template <typename T>
__device__ __forceinline__ T interp(const T* e, Dims c, int i, int j, int k) {
    const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
    const int I1 = (i & 1) ? wrapc(I0 + 1, c.n1) : I0;
    const int J1 = (j & 1) ? wrapc(J0 + 1, c.n2) : J0;
    const int K1 = (k & 1) ? wrapc(K0 + 1, c.n3) : K0;
    // (1 - w) is the weight of the second node; for even indices both nodes coincide
    const float wx = (i & 1) ? 0.5f : 1.0f, wy = (j & 1) ? 0.5f : 1.0f, wz = (k & 1) ? 0.5f : 1.0f;
    auto at = [&](int I, int J, int K) { return e[((long long)K * c.n2 + J) * c.n1 + I]; };
    auto lx = [&](int J, int K) { return vfma(wx, at(I0, J, K), vmul(1.f - wx, at(I1, J, K))); };
    auto ly = [&](int K) { return vfma(wy, lx(J0, K), vmul(1.f - wy, lx(J1, K))); };
    return vfma(wz, ly(K0), vmul(1.f - wz, ly(K1)));
}

// fine x += trilinear interpolation of coarse e
template <typename T>
__global__ void k_prolong_add(Dims f, Dims c, const T* __restrict__ e, T* __restrict__ x,
                              const double* done) {
    pdl_enter();
    if (*done != 0.0) return;
    // 3-D launch (x_blocks, y_blocks, f.n3) of 32 x 8 threads: no index division
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= f.n1 || j >= f.n2) return;
    const long long idx = ((long long)k * f.n2 + j) * f.n1 + i;
    x[idx] = vadd(x[idx], interp(e, c, i, j, k));
}

// ---- the small levels inside one thread-block cluster (second-order operator on all of them)
struct SmallLevels {
    int count;
    int solo;     // levels solo .. count - 1 run on the cluster's first CTA alone
    int deg;
    int deg_coarse;
    float ctheta, cdelta;
    float sigma;
    Dims d[MG_MAX_LEVELS];
    float cx[MG_MAX_LEVELS], cy[MG_MAX_LEVELS], cz[MG_MAX_LEVELS], centre[MG_MAX_LEVELS];
    float invD[MG_MAX_LEVELS], theta[MG_MAX_LEVELS];
    float ca[MG_MAX_LEVELS][4], cb[MG_MAX_LEVELS][4];
    void *x[MG_MAX_LEVELS], *b[MG_MAX_LEVELS], *r[MG_MAX_LEVELS];
    void *dv[MG_MAX_LEVELS], *dw[MG_MAX_LEVELS];   // the Chebyshev direction, double-buffered
    int soff[MG_MAX_LEVELS];   // solo levels: element offset of their arrays in shared memory
};

// The five arrays of level l: x, b, r and the two direction buffers (k = 0..4).  Solo levels
// keep them in the first CTA's shared memory (five consecutive runs of n_l elements from
// soff[l]), the others in global memory.
template <typename T, bool SOLO>
__device__ __forceinline__ T* lv_arr(const SmallLevels& P, int l, int k) {
    if constexpr (SOLO) {
        extern __shared__ float4 mg_solo_smem[];
        return reinterpret_cast<T*>(mg_solo_smem) + P.soff[l] + (long long)k * P.d[l].n;
    } else {
        void* p = k == 0 ? P.x[l] : k == 1 ? P.b[l] : k == 2 ? P.r[l] : k == 3 ? P.dv[l] : P.dw[l];
        return reinterpret_cast<T*>(p);
    }
}

// -(A a)(i) = (L_h a)(i) - sigma a(i) for the 7-point operator of level l
template <typename T>
__device__ __forceinline__ T neg_op7(const SmallLevels& P, int l, const T* a, int i) {
    const Dims& d = P.d[l];
    const int ix = i % d.n1, iy = (i / d.n1) % d.n2, iz = i / (d.n1 * d.n2);
    const int sx = d.n1, sy = d.n1 * d.n2;
    T v = vmul(P.centre[l] - P.sigma, a[i]);
    v = vfma(P.cx[l], vadd(a[i - ix + wrapc(ix + 1, d.n1)], a[i - ix + wrapc(ix - 1, d.n1)]), v);
    v = vfma(P.cy[l], vadd(a[i + (wrapc(iy + 1, d.n2) - iy) * sx], a[i + (wrapc(iy - 1, d.n2) - iy) * sx]), v);
    v = vfma(P.cz[l], vadd(a[i + (wrapc(iz + 1, d.n3) - iz) * sy], a[i + (wrapc(iz - 1, d.n3) - iz) * sy]), v);
    return v;
}

// The small levels run on one thread-block cluster (MG_CLUSTER CTAs of 1024 threads, one per
// SM) that steps through the phases of the V-cycle with hardware cluster barriers.
constexpr int MG_CLUSTER = 8;

__device__ __forceinline__ int cl_tid() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int cl_stride() { return gridDim.x * blockDim.x; }
__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
// Levels of at most MG_SOLO_POINTS run on the first CTA alone with block barriers (a cluster
// barrier costs about a microsecond, several times the work of a sweep of such a level).
constexpr int MG_SOLO_POINTS = 4096;
template <bool SOLO> __device__ __forceinline__ int lv_tid() { return SOLO ? (int)threadIdx.x : cl_tid(); }
template <bool SOLO> __device__ __forceinline__ int lv_stride() { return SOLO ? (int)blockDim.x : cl_stride(); }
template <bool SOLO> __device__ __forceinline__ void lv_sync() {
    if (SOLO) __syncthreads();
    else cl_sync();
}

// Chebyshev smoothing of level l (zero initial guess, or starting from x): the whole cluster,
// or the first CTA alone (SOLO).  One barrier per step: step k reads the direction d_k at the
// neighbours and writes x, r and d_{k+1} of its own points, d_{k+1} into the other buffer.
// With a zero guess, d_0 = D^{-1} b / theta is already in dv (written by the restriction) when
// d0_ready, else formed here.
template <typename T, bool SOLO>
__device__ void blk_smooth(const SmallLevels& P, int l, bool zero, bool d0_ready) {
    const int n = (int)P.d[l].n;
    T *x = lv_arr<T, SOLO>(P, l, 0), *b = lv_arr<T, SOLO>(P, l, 1), *r = lv_arr<T, SOLO>(P, l, 2);
    T* dbuf[2] = {lv_arr<T, SOLO>(P, l, 3), lv_arr<T, SOLO>(P, l, 4)};
    const float s0 = P.invD[l] / P.theta[l];
    const int t0 = lv_tid<SOLO>(), ts = lv_stride<SOLO>();
    if (zero) {
        if (!d0_ready) {
            for (int i = t0; i < n; i += ts) dbuf[0][i] = vmul(s0, b[i]);
            lv_sync<SOLO>();
        }
    } else {
        for (int i = t0; i < n; i += ts) {
            const T rv = vadd(b[i], neg_op7(P, l, x, i));
            r[i] = rv;
            dbuf[0][i] = vmul(s0, rv);
        }
        lv_sync<SOLO>();
    }
    for (int k = 0; k < P.deg; ++k) {
        const bool first = zero && k == 0;
        const T* dc = dbuf[k & 1];
        T* dn = dbuf[(k + 1) & 1];
        const bool more = k + 1 < P.deg;
        const float ca = more ? P.ca[l][k] : 0.f, cb = more ? P.cb[l][k] * P.invD[l] : 0.f;
        for (int i = t0; i < n; i += ts) {
            const T di = dc[i];
            x[i] = first ? di : vadd(x[i], di);
            const T rv = vadd(first ? b[i] : r[i], neg_op7(P, l, dc, i));
            r[i] = rv;
            if (more) dn[i] = vfma(ca, di, vmul(cb, rv));
        }
        lv_sync<SOLO>();
    }
}

// coarse b[l + 1] = full weighting of r[l], and the first Chebyshev direction of level l + 1
// (its smoother's, or the coarse solve's) from it
template <typename T, bool SOLO>
__device__ void blk_restrict(const SmallLevels& P, int l) {
    const float w[3] = {0.25f, 0.5f, 0.25f};
    const Dims f = P.d[l], c = P.d[l + 1];
    const T* r = lv_arr<T, SOLO>(P, l, 2);
    T* bc = lv_arr<T, SOLO>(P, l + 1, 1);
    T* dc = lv_arr<T, SOLO>(P, l + 1, 3);
    const float s0 = P.invD[l + 1] / (l + 2 == P.count ? P.ctheta : P.theta[l + 1]);
    for (int I = lv_tid<SOLO>(); I < (int)c.n; I += lv_stride<SOLO>()) {
        const int ci = I % c.n1, cj = (I / c.n1) % c.n2, ck = I / (c.n1 * c.n2);
        T s = vzero<T>();
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int fx = wrapc(2 * ci + dx, f.n1), fy = wrapc(2 * cj + dy, f.n2),
                              fz = wrapc(2 * ck + dz, f.n3);
                    s = vfma(w[dz + 1] * w[dy + 1] * w[dx + 1], r[(fz * f.n2 + fy) * f.n1 + fx], s);
                }
        bc[I] = s;
        dc[I] = vmul(s0, s);
    }
    lv_sync<SOLO>();
}

// x[l] += interpolation of x[l + 1]
template <typename T, bool SOLO>
__device__ void blk_prolong(const SmallLevels& P, int l) {
    const Dims f = P.d[l], c = P.d[l + 1];
    const T* e = lv_arr<T, SOLO>(P, l + 1, 0);
    T* x = lv_arr<T, SOLO>(P, l, 0);
    for (int i = lv_tid<SOLO>(); i < (int)f.n; i += lv_stride<SOLO>()) {
        const int fi = i % f.n1, fj = (i / f.n1) % f.n2, fk = i / (f.n1 * f.n2);
        x[i] = vadd(x[i], interp(e, c, fi, fj, fk));
    }
    lv_sync<SOLO>();
}

// coarsest level: Chebyshev over the whole spectrum (non-zero part for sigma = 0) from zero;
// the first direction D^{-1} b / theta comes from the restriction when d0_ready.  One barrier
// per step, as in blk_smooth.
template <typename T, bool SOLO>
__device__ void blk_coarse(const SmallLevels& P, bool d0_ready) {
    const int l = P.count - 1;
    const int n = (int)P.d[l].n;
    T *x = lv_arr<T, SOLO>(P, l, 0), *b = lv_arr<T, SOLO>(P, l, 1), *r = lv_arr<T, SOLO>(P, l, 2);
    T* dbuf[2] = {lv_arr<T, SOLO>(P, l, 3), lv_arr<T, SOLO>(P, l, 4)};
    const float sigma1 = P.ctheta / P.cdelta;
    float rho = 1.f / sigma1;
    const int t0 = lv_tid<SOLO>(), ts = lv_stride<SOLO>();
    if (!d0_ready) {
        for (int i = t0; i < n; i += ts) dbuf[0][i] = vmul(P.invD[l] / P.ctheta, b[i]);
        lv_sync<SOLO>();
    }
    for (int s = 0; s < P.deg_coarse; ++s) {
        const float rn = 1.f / (2.f * sigma1 - rho);
        const float a = rn * rho, bb = 2.f * rn / P.cdelta * P.invD[l];
        const T* dc = dbuf[s & 1];
        T* dn = dbuf[(s + 1) & 1];
        for (int i = t0; i < n; i += ts) {
            const T di = dc[i];
            x[i] = s == 0 ? di : vadd(x[i], di);
            const T rv = vadd(s == 0 ? b[i] : r[i], neg_op7(P, l, dc, i));
            r[i] = rv;
            dn[i] = vfma(a, di, vmul(bb, rv));
        }
        lv_sync<SOLO>();
        rho = rn;
    }
}

// Levels solo .. count - 1 on the first CTA alone, in its shared memory: b of the first solo
// level (and its first direction, when the cluster's restriction formed it) come in from
// global memory, its x goes back out for the cluster's prolongation.
template <typename T>
__device__ void solo_part(const SmallLevels& P) {
    const int s0 = P.solo;
    const int n0 = (int)P.d[s0].n;
    const T* gb = (const T*)P.b[s0];
    const T* gd = (const T*)P.dv[s0];
    T* sb = lv_arr<T, true>(P, s0, 1);
    T* sd = lv_arr<T, true>(P, s0, 3);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        sb[i] = gb[i];
        if (s0 > 0) sd[i] = gd[i];
    }
    __syncthreads();
    for (int l = s0; l + 1 < P.count; ++l) {
        blk_smooth<T, true>(P, l, true, l > 0);
        blk_restrict<T, true>(P, l);
    }
    blk_coarse<T, true>(P, P.count > 1);
    for (int l = P.count - 2; l >= s0; --l) {
        blk_prolong<T, true>(P, l);
        blk_smooth<T, true>(P, l, false, false);
    }
    const T* sx = lv_arr<T, true>(P, s0, 0);
    T* gx = (T*)P.x[s0];
    for (int i = threadIdx.x; i < n0; i += blockDim.x) gx[i] = sx[i];
}

template <typename T>
__global__ void __cluster_dims__(MG_CLUSTER, 1, 1) __launch_bounds__(1024)
k_small_vcycle(SmallLevels P, const double* done) {
    pdl_enter();
    if (*done != 0.0) return;
    // every cluster barrier below is reached by all CTAs: the solo part contains none
    for (int l = 0; l < P.solo && l + 1 < P.count; ++l) {
        blk_smooth<T, false>(P, l, true, l > 0);
        blk_restrict<T, false>(P, l);
    }
    if (P.solo >= P.count) blk_coarse<T, false>(P, P.count > 1);
    else if (blockIdx.x == 0) solo_part<T>(P);
    for (int l = min(P.solo, P.count - 1) - 1; l >= 0; --l) {
        if (l + 1 == P.solo) cl_sync();   // the first CTA has finished the solo levels
        blk_prolong<T, false>(P, l);
        blk_smooth<T, false>(P, l, false, false);
    }
}

// Chebyshev coefficients for steps k = 0..deg-1 on [lmin, lmax]: returned as the pair
// (a_k, b_k) used to form d_{k+1} = a_k d_k + b_k D^{-1} r_{k+1}.
static void cheby_coeffs(double lmin, double lmax, int deg, std::vector<float>& a,
                         std::vector<float>& b, double& theta) {
    theta = 0.5 * (lmax + lmin);
    const double delta = 0.5 * (lmax - lmin);
    const double sigma1 = theta / delta;
    double rho = 1.0 / sigma1;
    a.resize(deg);
    b.resize(deg);
    for (int k = 0; k < deg; ++k) {
        const double rn = 1.0 / (2.0 * sigma1 - rho);
        a[k] = (float)(rn * rho);
        b[k] = (float)(2.0 * rn / delta);
        rho = rn;
    }
}

template <typename T>
static void smooth(of_grid* g, MGLevel& L, int deg, bool zero_guess, const double* done, double sigma,
                   const BetaFuse<T>* fuse = nullptr) {
    constexpr int RY = std::is_same<T, float>::value ? 2 : 1;
    const Shifted S = shifted_level(L, sigma);
    std::vector<float> a, b;
    double theta;
    cheby_coeffs(0.15 * S.lmax, 1.05 * S.lmax, deg, a, b, theta);
    T *x = (T*)L.x, *lb = (T*)L.b, *r = (T*)L.r;
    T* dbuf[2] = {(T*)L.d0, (T*)L.d1};
    const float s0 = (float)(S.invD / theta);
    // from a guess: r and the first direction s0 r (in dbuf[1], which step 0 reads; step 0
    // writes r in place, so it must not read r at the neighbours)
    if (!zero_guess)
        launch_stencil_dims<T, RY>(g, L.d, L.N, L.W, OpResid32<T>{x, lb, r, (float)sigma, done, dbuf[1], s0});
    for (int k = 0; k < deg; ++k) {
        OpCheby<T> op;
        op.din = (k == 0 && zero_guess) ? lb : dbuf[(k + 1) & 1];
        op.dscale = (k == 0 && zero_guess) ? s0 : 1.f;
        op.x = x;
        op.x_init = zero_guess && k == 0;
        op.rin = (k == 0 && zero_guess) ? lb : r;
        op.rout = r;
        op.dout = (k + 1 < deg) ? dbuf[k & 1] : nullptr;
        op.a = a[k];
        op.bD = b[k] * S.invD;
        op.sigma = (float)sigma;
        op.done = done;
        if (fuse && k + 1 == deg) {
            op.rk = fuse->r;
            op.st = fuse->st;
            op.rc = red_ctx(g, 0);
            op.first = fuse->first;
            op.n = L.d.n;
        }
        launch_stencil_dims<T, RY>(g, L.d, L.N, L.W, op);
    }
}

// z = M^{-1} r, one V-cycle for A = -L_h + sigma; r, z fine-level fields.  Levels above
// first_small are swept by grid-wide launches, the rest by k_small_vcycle on one cluster.
template <typename T>
static bool vcycle(of_grid* g, const T* r, T* z, const double* done, double sigma,
                   const BetaFuse<T>* fuse = nullptr) {
    MG& m = *g->mg;
    const int nl = (int)m.lv.size();
    const int fs = m.first_small;
    float* saved_b = m.lv[0].b;
    float* saved_x = m.lv[0].x;
    m.lv[0].b = (float*)const_cast<T*>(r);
    m.lv[0].x = (float*)z;
    for (int l = 0; l < fs; ++l) {
        MGLevel& L = m.lv[l];
        MGLevel& C = m.lv[l + 1];
        smooth<T>(g, L, m.deg, true, done, sigma);   // x_l = S b_l, r_l = b_l - A x_l
        ProfScope ps(g, PC_MG_TRANSFER, sizeof(T) * (double)(L.d.n + C.d.n));
        launch_pdl(k_restrict<T>, grid3(C.d), dim3(32, 8), 0, g->stream, L.d, C.d,
                   (const T*)L.r, (T*)C.b, done);
    }
    {
        SmallLevels P{};
        P.count = nl - fs;
        P.solo = P.count;
        while (P.solo > 0 && m.lv[fs + P.solo - 1].d.n <= MG_SOLO_POINTS) --P.solo;
        P.deg = m.deg;
        P.sigma = (float)sigma;
        const Shifted SC = shifted_level(m.lv[nl - 1], sigma);
        const double kappa = SC.lmax / std::max(SC.lmin, 1e-12);
        P.deg_coarse = std::min(96, std::max(8, (int)std::ceil(2.0 * std::sqrt(kappa))));
        P.ctheta = (float)(0.5 * (SC.lmax + SC.lmin));
        P.cdelta = (float)(0.5 * (SC.lmax - SC.lmin));
        for (int k = 0; k < P.count; ++k) {
            const MGLevel& L = m.lv[fs + k];
            const Shifted S = shifted_level(L, sigma);
            P.d[k] = L.d;
            P.cx[k] = L.W.w[0][1];
            P.cy[k] = L.W.w[1][1];
            P.cz[k] = L.W.w[2][1];
            P.centre[k] = L.W.centre;
            P.invD[k] = S.invD;
            std::vector<float> a, b;
            double theta;
            cheby_coeffs(0.15 * S.lmax, 1.05 * S.lmax, m.deg, a, b, theta);
            P.theta[k] = (float)theta;
            for (int j = 0; j < m.deg && j < 4; ++j) {
                P.ca[k][j] = a[j];
                P.cb[k][j] = b[j];
            }
            P.x[k] = L.x;
            P.b[k] = L.b;
            P.r[k] = L.r;
            P.dv[k] = L.d0;
            P.dw[k] = L.d1;
        }
        // shared memory of the solo levels: five arrays each
        size_t elems = 0;
        for (int k = P.solo; k < P.count; ++k) {
            P.soff[k] = (int)elems;
            elems += 5 * (size_t)P.d[k].n;
        }
        const size_t smem = (elems * sizeof(T) + 15) / 16 * 16;
        OF_REQUIRE(smem <= 227 * 1024, OF_EINVAL, "multigrid: %zu bytes of small levels exceed shared memory", smem);
        if (smem > 48 * 1024) {   // above the default limit: raise it (per host thread and device)
            static thread_local int configured_device = -1;
            static thread_local size_t configured = 0;
            if (configured_device != g->device || configured < smem) {
                OF_CUDA(cudaFuncSetAttribute(k_small_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024));
                configured_device = g->device;
                configured = 227 * 1024;
            }
        }
        ProfScope ps(g, PC_MG_TRANSFER, 0.0);
        launch_pdl(k_small_vcycle<T>, MG_CLUSTER, 1024, smem, g->stream, P, done);
    }
    for (int l = fs - 1; l >= 0; --l) {
        MGLevel& L = m.lv[l];
        MGLevel& C = m.lv[l + 1];
        {
            ProfScope ps(g, PC_MG_TRANSFER, sizeof(T) * (double)(2 * L.d.n + C.d.n));
            launch_pdl(k_prolong_add<T>, grid3(L.d), dim3(32, 8), 0, g->stream, L.d, C.d,
                       (const T*)C.x, (T*)L.x, done);
        }
        smooth<T>(g, L, m.deg, false, done, sigma, l == 0 ? fuse : nullptr);
    }
    m.lv[0].b = saved_b;
    m.lv[0].x = saved_x;
    return fs >= 1 && m.deg >= 1;   // the last sweep was level 0's, and carried the fusion
}

void mg_vcycle_real_shifted(of_grid* g, const float* r, float* z, const double* done, double sigma) {
    vcycle<float>(g, r, z, done, sigma);
}

void mg_vcycle(of_grid* g, const float* r, float* z, const double* done) {
    vcycle<float>(g, r, z, done, 0.0);
}

void mg_vcycle_shifted(of_grid* g, const float2* r, float2* z, const double* done, double sigma) {
    vcycle<float2>(g, r, z, done, sigma);
}

bool mg_vcycle_beta(of_grid* g, const float* r, float* z, KState* st, bool first) {
    const BetaFuse<float> f{st, first, r};
    return vcycle<float>(g, r, z, &st->done, 0.0, &f);
}

bool mg_vcycle_shifted_beta(of_grid* g, const float2* r, float2* z, KState* st, bool first, double sigma) {
    const BetaFuse<float2> f{st, first, r};
    return vcycle<float2>(g, r, z, &st->done, sigma, &f);
}

}  // namespace of
