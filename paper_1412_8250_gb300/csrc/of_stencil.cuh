// Order-2N periodic finite-difference Laplacian (Eq. FD:Laplacian, periodic wrap of Sec. 4)
// as a tiled sweep with pluggable load/store "ops", so that Krylov updates, Hamiltonian
// terms and reductions are fused into the same pass over the grid.
//
// Tiling: a block of 32 x 8 threads owns a 32 x (8*RY) tile of the x-y plane and marches
// along z through `cz` planes.  Each thread keeps the 2N+1 z-neighbours of its RY points in
// registers (a shifting queue); the x- and y-neighbours come from the current z-plane staged
// in shared memory with an N-point halo whose periodic indices are precomputed once per
// block.  Symmetric taps are paired: w_p (f(i+p) + f(i-p)).
#pragma once

#include <type_traits>
#include <utility>

#include "of_internal.cuh"

namespace of {

// ------------------------------------------------------------------ value arithmetic
// Real scalars (float, double) and interleaved complex (float2, double2) share the same
// real-weighted stencil arithmetic.
template <typename T> struct Real;
template <> struct Real<float> { using type = float; };
template <> struct Real<double> { using type = double; };
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ float vfma(float w, float a, float c) { return fmaf(w, a, c); }
__device__ __forceinline__ double vfma(double w, double a, double c) { return fma(w, a, c); }
__device__ __forceinline__ float2 vfma(float w, float2 a, float2 c) { return make_float2(fmaf(w, a.x, c.x), fmaf(w, a.y, c.y)); }
__device__ __forceinline__ double2 vfma(double w, double2 a, double2 c) { return make_double2(fma(w, a.x, c.x), fma(w, a.y, c.y)); }

__device__ __forceinline__ float vmul(float w, float a) { return w * a; }
__device__ __forceinline__ double vmul(double w, double a) { return w * a; }
__device__ __forceinline__ float2 vmul(float w, float2 a) { return make_float2(w * a.x, w * a.y); }
__device__ __forceinline__ double2 vmul(double w, double2 a) { return make_double2(w * a.x, w * a.y); }

__device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

constexpr int ST_BX = 32;
constexpr int ST_BY = 8;
constexpr int ST_THREADS = ST_BX * ST_BY;

// Op interface (all __device__):
//   bool begin()                         -- false: the whole kernel is a no-op (uniform)
//   T load(long long i) const            -- value of the differentiated field at i
//   void store(long long i, T c, T lap)  -- c = field at i, lap = (L_h field)(i)
//   void end()                           -- called by every thread of every active block
//
// Pipeline per z-plane (one barrier per plane): the x-y tile of plane z+1 (with its periodic
// halo) sits in registers, loaded one plane ahead; it is written to the free half of a
// double-buffered shared tile while plane z is computed from the other half.  The z
// neighbours of each thread's points shift through a register queue, whose newest entry
// (plane z+N) is also loaded one plane ahead.  In-plane offsets of the tile elements a
// thread loads are computed once per block.
// One block's share of a sweep: tile (bx, by) of the x-y plane, planes [bz*cz, bz*cz + cz).
template <typename T, int N, int RY, class Op>
__device__ __forceinline__ void stencil_tile(const Dims& d, const Weights<typename Real<T>::type>& W,
                                             int cz, int bx, int by, int bz, Op& op) {
    constexpr int TY = ST_BY * RY;
    constexpr int SX = ST_BX + 2 * N;
    constexpr int SY = TY + 2 * N;
    constexpr int TILE = SX * SY;
    constexpr int PER = (TILE + ST_THREADS - 1) / ST_THREADS;
    constexpr int Q = 2 * N + 1;
    __shared__ T tile[2][SY][SX];
    __shared__ int xi[SX];
    __shared__ int yi[SY];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ST_BX * ty;
    const int x0 = bx * ST_BX;
    const int y0 = by * TY;
    const int z0 = bz * cz;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    for (int t = tid; t < SX; t += ST_THREADS) xi[t] = wrap_index(x0 - N + t, n1);
    for (int t = tid; t < SY; t += ST_THREADS) yi[t] = wrap_index(y0 - N + t, n2);
    __syncthreads();

    const int x = x0 + tx;
    const bool xin = x < n1;
    const int xs = xi[tx + N];
    const long long plane = (long long)n1 * n2;
    long long rowoff[RY];
    bool yin[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int yl = ty + r * ST_BY;
        rowoff[r] = (long long)yi[yl + N] * n1 + xs;
        yin[r] = (y0 + yl) < n2;
    }
    int goff[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = tid + k * ST_THREADS;
        if (e < TILE) {
            const int sy = e / SX, sx = e - sy * SX;
            goff[k] = yi[sy] * n1 + xi[sx];
        } else {
            goff[k] = 0;
        }
    }
    T* tile0 = &tile[0][0][0];
    T* tile1 = &tile[1][0][0];

    T q[RY][Q];
    T pre[PER];
    T qn[RY];
    const int zend = min(z0 + cz, n3);
    if (z0 < n3) {
#pragma unroll
        for (int j = 0; j < 2 * N; ++j) {
            const long long zo = (long long)wrap_index(z0 - N + j, n3) * plane;
#pragma unroll
            for (int r = 0; r < RY; ++r) q[r][j] = op.load(zo + rowoff[r]);
        }
        {   // plane z0 straight into buffer 0; plane z0 + 1 and queue entry z0 + N into registers
            const long long zo = (long long)z0 * plane;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int e = tid + k * ST_THREADS;
                if (e < TILE) tile0[e] = op.load(zo + goff[k]);
            }
            const long long z1 = (long long)wrap_index(z0 + 1, n3) * plane;
#pragma unroll
            for (int k = 0; k < PER; ++k) pre[k] = op.load(z1 + goff[k]);
            const long long zq = (long long)wrap_index(z0 + N, n3) * plane;
#pragma unroll
            for (int r = 0; r < RY; ++r) qn[r] = op.load(zq + rowoff[r]);
        }
        __syncthreads();
        int buf = 0;
        for (int z = z0; z < zend; ++z) {
            T* cur = buf ? tile1 : tile0;
            T* nxt = buf ? tile0 : tile1;
#pragma unroll
            for (int r = 0; r < RY; ++r) q[r][2 * N] = qn[r];
            if (z + 1 < zend) {
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int e = tid + k * ST_THREADS;
                    if (e < TILE) nxt[e] = pre[k];
                }
                const long long z2 = (long long)wrap_index(z + 2, n3) * plane;
#pragma unroll
                for (int k = 0; k < PER; ++k) pre[k] = op.load(z2 + goff[k]);
                const long long zq = (long long)wrap_index(z + 1 + N, n3) * plane;
#pragma unroll
                for (int r = 0; r < RY; ++r) qn[r] = op.load(zq + rowoff[r]);
            }
            const long long zc = (long long)z * plane;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int ly = ty + r * ST_BY + N, lx = tx + N;
                const T c = q[r][N];
                T acc = vmul(W.centre, c);
#pragma unroll
                for (int p = 1; p <= N; ++p) {
                    acc = vfma(W.w[2][p], vadd(q[r][N + p], q[r][N - p]), acc);
                    acc = vfma(W.w[0][p], vadd(cur[ly * SX + lx + p], cur[ly * SX + lx - p]), acc);
                    acc = vfma(W.w[1][p], vadd(cur[(ly + p) * SX + lx], cur[(ly - p) * SX + lx]), acc);
                }
                if (xin && yin[r]) op.store(zc + (long long)(y0 + ty + r * ST_BY) * n1 + x, c, acc);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int j = 0; j < 2 * N; ++j) q[r][j] = q[r][j + 1];
            buf ^= 1;
        }
    }
}

// ---------------------------------------------------------------- FP32 fast path
// For FP32 fields with an even n1: a block of 16 x (32 / RY) threads owns a 32 x 32 tile of the
// x-y plane, each thread two x-neighbouring points (one float2) in RY adjacent rows, whose y
// taps share one column of staged values.  Every two-element chunk of the
// staged tile (with its periodic halo) starts at an even x and so is contiguous in global
// memory even where the halo wraps, so the tile moves as 64-bit loads and stores.  The z
// neighbours sit in a register queue of float2 rotated by compile-time index (the z loop is
// unrolled by 2N + 1), the z and y taps use packed FP32x2 arithmetic, the x taps scalar FP32.
constexpr int S2_BX = 16;    // threads in x (two points each)
constexpr int S2_TY = 32;    // rows per tile

template <class Op, class = void>
struct HasLoad2 { static constexpr bool value = false; };
template <class Op>
struct HasLoad2<Op, decltype((void)std::declval<const Op&>().load2(0LL), void())> {
    static constexpr bool value = true;
};
template <class Op>
__device__ __forceinline__ float2 op_load2(const Op& op, long long i) {
    if constexpr (HasLoad2<Op>::value) return op.load2(i);
    else return make_float2(op.load(i), op.load(i + 1));
}

__device__ __forceinline__ unsigned long long pk2(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
// packed FP32x2: a + b, and w (both lanes) * s + c
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long w, unsigned long long s,
                                                   unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w), "l"(s), "l"(c));
    return r;
}

template <int N, int RY, class Op>
__device__ __forceinline__ void stencil2_tile(const Dims& d, const Weights<float>& W, int cz, int bx,
                                              int by, int bz, Op& op) {
    constexpr int BY = S2_TY / RY;            // threads in y
    constexpr int THREADS = S2_BX * BY;
    constexpr int HX = (N + 1) & ~1;          // x halo, rounded up to even
    constexpr int TX = 2 * S2_BX;             // 32 points in x
    constexpr int SX = TX + 2 * HX;
    constexpr int SY = S2_TY + 2 * N;
    constexpr int C2 = SX / 2;                // two-element chunks per staged row
    constexpr int CH = C2 * SY;
    constexpr int PER = (CH + THREADS - 1) / THREADS;
    constexpr int Q = 2 * N + 1;
    __shared__ __align__(16) float tile[2][SY * SX];
    __shared__ int xi2[C2];
    __shared__ int yi[SY];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + S2_BX * ty;
    const int x0 = bx * TX, y0 = by * S2_TY, z0 = bz * cz;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    for (int t = tid; t < C2; t += THREADS) xi2[t] = wrap_index(x0 - HX + 2 * t, n1);
    for (int t = tid; t < SY; t += THREADS) yi[t] = wrap_index(y0 - N + t, n2);
    __syncthreads();

    // this thread's points: x, x + 1 in rows y0 + RY ty + r, r < RY
    const int x = x0 + 2 * tx;
    const long long plane = (long long)n1 * n2;
    long long rowoff[RY];
    bool act[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int yl = RY * ty + r;
        rowoff[r] = (long long)yi[yl + N] * n1 + (x < n1 ? x : 0);
        act[r] = x < n1 && y0 + yl < n2;      // n1 even: x + 1 < n1 as well
    }
    long long goff[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = tid + k * THREADS;
        const int sy = e / C2, c2 = e - (e / C2) * C2;
        goff[k] = e < CH ? (long long)yi[sy] * n1 + xi2[c2] : 0;
    }
    unsigned long long wz2[N + 1], wy2[N + 1];
#pragma unroll
    for (int p = 0; p <= N; ++p) {
        wz2[p] = pk2(make_float2(W.w[2][p], W.w[2][p]));
        wy2[p] = pk2(make_float2(W.w[1][p], W.w[1][p]));
    }
    const unsigned long long centre2 = pk2(make_float2(W.centre, W.centre));

    unsigned long long q[RY][Q];
    float2 pre[PER];
    float2 qn[RY];
    const int zend = min(z0 + cz, n3);
    if (z0 >= n3) return;
#pragma unroll
    for (int j = 0; j < 2 * N; ++j) {
        const long long zo = (long long)wrap_index(z0 - N + j, n3) * plane;
#pragma unroll
        for (int r = 0; r < RY; ++r) q[r][j] = pk2(op_load2(op, zo + rowoff[r]));
    }
    {
        const long long zo = (long long)z0 * plane;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * THREADS;
            if (e < CH) *reinterpret_cast<float2*>(&tile[0][2 * e]) = op_load2(op, zo + goff[k]);
        }
        const long long z1 = (long long)wrap_index(z0 + 1, n3) * plane;
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (tid + k * THREADS < CH) pre[k] = op_load2(op, z1 + goff[k]);
        const long long zq = (long long)wrap_index(z0 + N, n3) * plane;
#pragma unroll
        for (int r = 0; r < RY; ++r) qn[r] = op_load2(op, zq + rowoff[r]);
    }
    __syncthreads();
    const int ly0 = RY * ty + N, lx = HX + 2 * tx;
    // running offsets of planes z + 2 and z + 1 + N, wrapped by one subtraction (both start
    // inside [0, n3) and advance by one plane per step)
    const long long wrapoff = (long long)n3 * plane;
    long long off_pre = (long long)wrap_index(z0 + 2, n3) * plane;
    long long off_q = (long long)wrap_index(z0 + 1 + N, n3) * plane;
    for (int zb = z0; zb < zend; zb += Q) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int z = zb + k;
            if (z >= zend) break;
            const int par = (z - z0) & 1;
            float* cur = tile[par];
            float* nxt = tile[par ^ 1];
#pragma unroll
            for (int r = 0; r < RY; ++r) q[r][(2 * N + k) % Q] = pk2(qn[r]);
            if (z + 1 < zend) {
#pragma unroll
                for (int kk = 0; kk < PER; ++kk) {
                    const int e = tid + kk * THREADS;
                    if (e < CH) *reinterpret_cast<float2*>(&nxt[2 * e]) = pre[kk];
                }
#pragma unroll
                for (int kk = 0; kk < PER; ++kk)
                    if (tid + kk * THREADS < CH) pre[kk] = op_load2(op, off_pre + goff[kk]);
#pragma unroll
                for (int r = 0; r < RY; ++r) qn[r] = op_load2(op, off_q + rowoff[r]);
            }
            off_pre += plane;
            if (off_pre >= wrapoff) off_pre -= wrapoff;
            off_q += plane;
            if (off_q >= wrapoff) off_q -= wrapoff;
            // z taps and centre
            unsigned long long acc[RY];
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                acc[r] = fma2(centre2, q[r][(N + k) % Q], 0ull);
#pragma unroll
                for (int p = 1; p <= N; ++p)
                    acc[r] = fma2(wz2[p], add2(q[r][(N + p + k) % Q], q[r][(N - p + k) % Q]), acc[r]);
            }
            // y taps: rows ly0 - N .. ly0 + RY - 1 + N of this column, each read once
            unsigned long long col[RY + 2 * N];
#pragma unroll
            for (int j = 0; j < RY + 2 * N; ++j)
                col[j] = pk2(*reinterpret_cast<const float2*>(&cur[(ly0 - N + j) * SX + lx]));
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int p = 1; p <= N; ++p)
                    acc[r] = fma2(wy2[p], add2(col[N + r + p], col[N + r - p]), acc[r]);
            // x taps, scalar, row by row
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                float v[2 * HX + 2];   // row ly0 + r, points lx - HX .. lx + 1 + HX
#pragma unroll
                for (int m = 0; m <= HX; ++m) {
                    const float2 t2 = *reinterpret_cast<const float2*>(&cur[(ly0 + r) * SX + lx - HX + 2 * m]);
                    v[2 * m] = t2.x;
                    v[2 * m + 1] = t2.y;
                }
                float2 a = upk2(acc[r]);
#pragma unroll
                for (int p = 1; p <= N; ++p) {
                    a.x = fmaf(W.w[0][p], v[HX + p] + v[HX - p], a.x);
                    a.y = fmaf(W.w[0][p], v[HX + 1 + p] + v[HX + 1 - p], a.y);
                }
                if (act[r]) {
                    const float2 c = upk2(q[r][(N + k) % Q]);
                    const long long i = (long long)z * plane + rowoff[r];
                    op.store(i, c.x, a.x);
                    op.store(i + 1, c.y, a.y);
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- FP32 brick kernel
// For FP32 fields (real, or complex as float2) on grids too small for long z runs (below 2^21
// points): a block of 16 x 8 threads owns a brick of 16 units x 8 rows x BZ planes, a unit
// being two x-neighbouring real points or one complex point, one float2 either way.  The brick
// and its periodic halo (N planes below and above, N rows, at least N points each side in x)
// are staged once into shared memory in 16-byte chunks, which stay contiguous across the
// periodic wrap (real n1 a multiple of 4, complex n1 even); each thread then holds the column
// of its unit through all BZ + 2N planes in registers for the z taps and reads its y and x
// taps from shared memory.  Every block is independent: no z-queue prologue and one barrier
// between staging and arithmetic, so that a 96^3 grid gives 432 (real) or 864 (complex)
// blocks with all staging loads in flight at once.
constexpr int B3_UX = 16;    // units (float2) per row of a brick = threads in x
constexpr int B3_BY = 8;     // rows per brick = threads in y
constexpr int B3_THREADS = B3_UX * B3_BY;

template <class Op, class = void>
struct HasStore2 { static constexpr bool value = false; };
template <class Op>
struct HasStore2<Op, decltype((void)std::declval<Op&>().store2(0LL, float2{}, float2{}), void())> {
    static constexpr bool value = true;
};
// two x-neighbouring real points i, i + 1 (i even)
template <class Op>
__device__ __forceinline__ void op_store2(Op& op, long long i, float2 c, float2 lap) {
    if constexpr (HasStore2<Op>::value) {
        op.store2(i, c, lap);
    } else {
        op.store(i, c.x, lap.x);
        op.store(i + 1, c.y, lap.y);
    }
}

// 16 bytes of the differentiated field from float offset f (a multiple of 4) of the grid
template <typename T, class Op>
__device__ __forceinline__ float4 brick_load4(const Op& op, long long f) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 a = op_load2(op, f), b = op_load2(op, f + 2);
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        const float2 a = op.load(f >> 1), b = op.load((f >> 1) + 1);
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

template <typename T, int N, int BZ, class Op>
__device__ __forceinline__ void brick_tile(const Dims& d, const Weights<float>& W, Op& op) {
    constexpr bool CPLX = std::is_same<T, float2>::value;
    constexpr int HXF = CPLX ? ((2 * N + 3) & ~3) : ((N + 3) & ~3);   // halo floats per side
    constexpr int HXC = HXF / 4;              // halo chunks per side
    constexpr int RW = 32 + 2 * HXF;          // floats per staged row of a central plane
    constexpr int ROWS = B3_BY + 2 * N;       // staged rows of a central plane
    constexpr int CPL = ROWS * RW;            // floats per central plane
    constexpr int ZP = BZ + 2 * N;            // planes of a unit's column
    constexpr int ZPL = B3_BY * 32;           // floats per z-halo plane (core rows only)
    constexpr int SLOTS = ROWS * 8 + B3_BY * 2 * HXC;   // chunks per central plane
    constexpr int SPT = (SLOTS + B3_THREADS - 1) / B3_THREADS;
    static_assert(B3_THREADS % 64 == 0, "z-halo staging assumes 64 chunks per plane");
    extern __shared__ float4 brick_smem[];    // central planes, then the z-halo planes
    float* cen = reinterpret_cast<float*>(brick_smem);
    float* zh = cen + BZ * CPL;
    __shared__ long long zoff[ZP];            // float offset of staged plane z0 - N + t
    __shared__ long long yoff[ROWS];          // float offset of staged row y0 - N + t in a plane
    __shared__ int xoff[RW / 4];              // float offset of staged chunk t in a row

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + B3_UX * ty;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    const int RF = CPLX ? 2 * n1 : n1;        // floats per grid row
    const long long PF = (long long)RF * n2;  // floats per grid plane
    const int x0f = blockIdx.x * 32, y0 = blockIdx.y * B3_BY, z0 = blockIdx.z * BZ;
    for (int t = tid; t < ZP; t += B3_THREADS) zoff[t] = (long long)wrap_index(z0 - N + t, n3) * PF;
    for (int t = tid; t < ROWS; t += B3_THREADS) yoff[t] = (long long)wrap_index(y0 - N + t, n2) * RF;
    for (int t = tid; t < RW / 4; t += B3_THREADS) xoff[t] = wrap_index(x0f - HXF + 4 * t, RF);
    __syncthreads();

    // central planes: each thread's chunk slots (row, chunk) are the same in every plane
#pragma unroll
    for (int m = 0; m < SPT; ++m) {
        const int sl = tid + m * B3_THREADS;
        if (sl < SLOTS) {
            int row, cc;
            if (sl < ROWS * 8) {
                row = sl >> 3;
                cc = HXC + (sl & 7);
            } else {
                const int s2 = sl - ROWS * 8;
                const int h = s2 % (2 * HXC);
                row = N + s2 / (2 * HXC);
                cc = h < HXC ? h : h + 8;
            }
            const long long go = yoff[row] + xoff[cc];
            float* so = cen + row * RW + 4 * cc;
            float4 v[BZ];
#pragma unroll
            for (int k = 0; k < BZ; ++k) v[k] = brick_load4<T>(op, zoff[N + k] + go);
#pragma unroll
            for (int k = 0; k < BZ; ++k) *reinterpret_cast<float4*>(so + k * CPL) = v[k];
        }
    }
    {   // z-halo planes j < N (z0 - N + j) and j >= N (z0 + BZ + j - N): core rows only
        const int sl = tid & 63, j0 = tid >> 6;
        const int row = sl >> 3, cc = HXC + (sl & 7);
        const long long go = yoff[N + row] + xoff[cc];
        float* so = zh + row * 32 + 4 * (sl & 7);
        constexpr int JP = B3_THREADS / 64;
        constexpr int NJ = (2 * N + JP - 1) / JP;
        float4 v[NJ];
#pragma unroll
        for (int m = 0; m < NJ; ++m) {
            const int j = j0 + m * JP;
            if (j < 2 * N) v[m] = brick_load4<T>(op, zoff[j < N ? j : j + BZ] + go);
        }
#pragma unroll
        for (int m = 0; m < NJ; ++m) {
            const int j = j0 + m * JP;
            if (j < 2 * N) *reinterpret_cast<float4*>(so + j * ZPL) = v[m];
        }
    }
    __syncthreads();

    // this thread's unit: floats 2 tx, 2 tx + 1 of row ty; its column through the ZP planes
    const int uo = 2 * tx;
    unsigned long long col[ZP];
#pragma unroll
    for (int j = 0; j < ZP; ++j) {
        const float* src = j < N ? zh + j * ZPL + ty * 32 + uo
                         : j < N + BZ ? cen + (j - N) * CPL + (ty + N) * RW + HXF + uo
                                      : zh + (j - BZ) * ZPL + ty * 32 + uo;
        col[j] = pk2(*reinterpret_cast<const float2*>(src));
    }
    unsigned long long wz2[N + 1], wy2[N + 1], wx2[N + 1];
#pragma unroll
    for (int p = 0; p <= N; ++p) {
        wz2[p] = pk2(make_float2(W.w[2][p], W.w[2][p]));
        wy2[p] = pk2(make_float2(W.w[1][p], W.w[1][p]));
        wx2[p] = pk2(make_float2(W.w[0][p], W.w[0][p]));
    }
    const unsigned long long centre2 = pk2(make_float2(W.centre, W.centre));
    const int y = y0 + ty;
    const int xu = (x0f >> 1) + tx;           // complex: point index; real: x / 2
    const bool act = y < n2 && (CPLX ? xu < n1 : 2 * xu < n1);
    const long long rowi = (long long)y * n1 + (CPLX ? xu : 2 * xu);   // grid index in units of T
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        const int z = z0 + k;
        if (z >= n3) break;
        unsigned long long acc = fma2(centre2, col[N + k], 0ull);
#pragma unroll
        for (int p = 1; p <= N; ++p) acc = fma2(wz2[p], add2(col[N + k + p], col[N + k - p]), acc);
        const float* b = cen + k * CPL + (ty + N) * RW + HXF + uo;
#pragma unroll
        for (int p = 1; p <= N; ++p)
            acc = fma2(wy2[p], add2(pk2(*reinterpret_cast<const float2*>(b + p * RW)),
                                    pk2(*reinterpret_cast<const float2*>(b - p * RW))), acc);
        if constexpr (CPLX) {
#pragma unroll
            for (int p = 1; p <= N; ++p)
                acc = fma2(wx2[p], add2(pk2(*reinterpret_cast<const float2*>(b + 2 * p)),
                                        pk2(*reinterpret_cast<const float2*>(b - 2 * p))), acc);
        } else {
            constexpr int HX = (N + 1) & ~1;  // row floats uo - HX .. uo + 1 + HX, in pairs
            float v[2 * HX + 2];
#pragma unroll
            for (int m = 0; m <= HX; ++m) {
                const float2 t2 = *reinterpret_cast<const float2*>(b - HX + 2 * m);
                v[2 * m] = t2.x;
                v[2 * m + 1] = t2.y;
            }
            float2 a = upk2(acc);
#pragma unroll
            for (int p = 1; p <= N; ++p) {
                a.x = fmaf(W.w[0][p], v[HX + p] + v[HX - p], a.x);
                a.y = fmaf(W.w[0][p], v[HX + 1 + p] + v[HX + 1 - p], a.y);
            }
            acc = pk2(a);
        }
        if (act) {
            const long long i = (long long)z * n2 * n1 + rowi;
            if constexpr (CPLX) op.store(i, upk2(col[N + k]), upk2(acc));
            else op_store2(op, i, upk2(col[N + k]), upk2(acc));
        }
    }
}

// dynamic shared memory of brick_tile: BZ central planes and 2N z-halo planes
template <typename T, int N, int BZ>
constexpr size_t brick_smem_bytes() {
    constexpr bool CPLX = std::is_same<T, float2>::value;
    constexpr int HXF = CPLX ? ((2 * N + 3) & ~3) : ((N + 3) & ~3);
    return sizeof(float) * ((size_t)BZ * (B3_BY + 2 * N) * (32 + 2 * HXF) + (size_t)2 * N * B3_BY * 32);
}

template <typename T, int N, int BZ, class Op>
__global__ void __launch_bounds__(B3_THREADS, 4) brick_kernel(Dims d, Weights<float> W, Op op) {
    pdl_enter();
    if (!op.begin()) return;
    brick_tile<T, N, BZ, Op>(d, W, op);
    op.end();
}

// planes per brick: 8 for the order-12 operator, 2 for the 7-point one (coarse levels, where
// a deeper brick leaves too few blocks)
template <int N> struct BrickDepth { static constexpr int value = N >= 3 ? 8 : 2; };

template <int N, int RY, class Op>
__global__ void __launch_bounds__(S2_BX * (S2_TY / RY), 2)
stencil2_kernel(Dims d, Weights<float> W, int cz, Op op) {
    pdl_enter();
    if (!op.begin()) return;
    stencil2_tile<N, RY, Op>(d, W, cz, blockIdx.x, blockIdx.y, blockIdx.z, op);
    op.end();
}

template <typename T, int N, int RY, class Op>
__global__ void __launch_bounds__(ST_THREADS)
stencil_kernel(Dims d, Weights<typename Real<T>::type> W, int cz, Op op) {
    pdl_enter();
    if (!op.begin()) return;
    stencil_tile<T, N, RY, Op>(d, W, cz, blockIdx.x, blockIdx.y, blockIdx.z, op);
    op.end();
}

// Launch geometry: z chunk chosen so the grid has at least ~4 blocks per SM when possible.
struct StencilLaunch {
    dim3 grid;
    int cz;
};

inline StencilLaunch stencil_launch(const Dims& d, int RY, int num_sms) {
    const int TY = ST_BY * RY;
    const int bx = (d.n1 + ST_BX - 1) / ST_BX;
    const int by = (d.n2 + TY - 1) / TY;
    const long long target = 4LL * num_sms;
    long long tiles = (long long)bx * by;
    int cz = (int)((d.n3 * tiles + target - 1) / target);
    if (cz < 1) cz = 1;
    if (cz > d.n3) cz = d.n3;
    if (cz < 4 && d.n3 >= 4) cz = 4;   // keep the z-halo overhead bounded
    int bz = (d.n3 + cz - 1) / cz;
    return {dim3(bx, by, bz), cz};
}

int num_sms();

// Profiling class and algorithmic words moved per point of a stencil op (defaults for plain
// Laplacian-like ops: read x, write y).
template <class Op, class = void>
struct OpInfo {
    static constexpr int cls = -1;
    static constexpr int words = 2;
};
template <class Op>
struct OpInfo<Op, decltype((void)Op::kClass, void())> {
    static constexpr int cls = Op::kClass;
    static constexpr int words = Op::kWords;
};

template <typename T, int N, class Op>
void launch_brick(of_grid* g, dim3 grid, dim3 block, const Dims& d, const Weights<float>& W, Op op) {
    constexpr int BZ = BrickDepth<N>::value;
    constexpr size_t smem = brick_smem_bytes<T, N, BZ>();
    // near or above the default 48 KB limit, which counts the op's static shared memory (its
    // reduction buffers) too: raise it once per thread
    if constexpr (smem > 40 * 1024) {
        static thread_local int configured_device = -1;
        if (configured_device != g->device) {
            OF_CUDA(cudaFuncSetAttribute(brick_kernel<T, N, BZ, Op>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            configured_device = g->device;
        }
    }
    launch_pdl(brick_kernel<T, N, BZ, Op>, grid, block, smem, g->stream, d, W, op);
}

template <typename T, int RY, class Op>
void launch_stencil_dims(of_grid* g, const Dims& d, int N,
                         const Weights<typename Real<T>::type>& W, Op op) {
    StencilLaunch sl = stencil_launch(d, RY, num_sms());
    dim3 block(ST_BX, ST_BY, 1);
    const int cls = OpInfo<Op>::cls >= 0 ? OpInfo<Op>::cls
                                         : (sizeof(typename Real<T>::type) == 8 ? PC_STENCIL_F64 : PC_STENCIL_F32);
    ProfScope ps(g, cls, (double)OpInfo<Op>::words * sizeof(T) * (double)d.n);
    cudaStream_t stream = g->stream;
    if constexpr (std::is_same<T, float>::value || std::is_same<T, float2>::value) {
        // FP32 brick kernel on small grids (order 12 and the 7-point coarse operator)
        constexpr bool CPLX = std::is_same<T, float2>::value;
        const long long RF = CPLX ? 2LL * d.n1 : d.n1;
        if (d.n < (1LL << 21) && (N == 6 || N == 1) && RF % 4 == 0) {
            const int bz = N == 6 ? BrickDepth<6>::value : BrickDepth<1>::value;
            const dim3 g3((unsigned)((RF + 31) / 32), (unsigned)((d.n2 + B3_BY - 1) / B3_BY),
                          (unsigned)((d.n3 + bz - 1) / bz));
            if ((long long)g3.x * g3.y * g3.z <= OF_MAX_RED_BLOCKS) {
                const dim3 b3(B3_UX, B3_BY, 1);
                if (N == 6) launch_brick<T, 6, Op>(g, g3, b3, d, W, op);
                else launch_brick<T, 1, Op>(g, g3, b3, d, W, op);
                return;
            }
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        // FP32 fast path on large grids: below ~128^3 points its 32 x 32 tiles leave too few
        // blocks to fill the GPU, and for the 7-point operator of the coarse multigrid levels
        // the smaller tiles of the general kernel are faster
        if (d.n1 % 2 == 0 && N == 6 && d.n >= (1LL << 21)) {
            const int bx = (d.n1 + 2 * S2_BX - 1) / (2 * S2_BX);
            const int by = (d.n2 + S2_TY - 1) / S2_TY;
            const long long tiles = (long long)bx * by;
            // one wave of two blocks per SM: as many z chunks as fit, at least 8 planes each
            const long long chunks = std::max(1LL, (2LL * num_sms()) / tiles);
            int cz = (int)((d.n3 + chunks - 1) / chunks);
            cz = std::max(cz, std::min(8, d.n3));
            constexpr int RY2 = 2;
            const dim3 grid2(bx, by, (d.n3 + cz - 1) / cz);
            const dim3 block2(S2_BX, S2_TY / RY2, 1);
            switch (N) {
                case 1: launch_pdl(stencil2_kernel<1, RY2, Op>, grid2, block2, 0, stream, d, W, cz, op); return;
                case 3: launch_pdl(stencil2_kernel<3, RY2, Op>, grid2, block2, 0, stream, d, W, cz, op); return;
                case 6: launch_pdl(stencil2_kernel<6, RY2, Op>, grid2, block2, 0, stream, d, W, cz, op); return;
                default: break;
            }
        }
    }
    switch (N) {
        case 1: launch_pdl(stencil_kernel<T, 1, RY, Op>, sl.grid, block, 0, stream, d, W, sl.cz, op); break;
        case 3: launch_pdl(stencil_kernel<T, 3, RY, Op>, sl.grid, block, 0, stream, d, W, sl.cz, op); break;
        case 6: launch_pdl(stencil_kernel<T, 6, RY, Op>, sl.grid, block, 0, stream, d, W, sl.cz, op); break;
        default: OF_REQUIRE(false, OF_EINVAL, "unsupported finite-difference half order %d", N);
    }
}

template <typename T, int RY, class Op>
void launch_stencil(of_grid* g, const Weights<typename Real<T>::type>& W, Op op) {
    launch_stencil_dims<T, RY, Op>(g, g->d, g->N, W, op);
}

inline int stencil_blocks(of_grid* g, int RY) {
    StencilLaunch sl = stencil_launch(g->d, RY, num_sms());
    return (int)(sl.grid.x * sl.grid.y * sl.grid.z);
}

// Reduction context handed to fused ops.
struct RedCtx {
    double* partials;
    unsigned int* counter;
    double* out;
};

inline RedCtx red_ctx(of_grid* g, int out_index) {
    return RedCtx{g->s.partials, g->s.counter, g->s.scalars + out_index};
}

// sum of a[i] * (b ? b[i] : 1) over i < n into rc.out[0] (defined in of_krylov.cu)
__global__ void k_sum_product(long long n, const double* a, const double* b, RedCtx rc);

// cached CUDA graphs of the Krylov solvers (of_krylov.cu)
void destroy_graphs(void* graphs);

// multigrid preconditioner (of_mg.cu): z = one V-cycle applied to r (FP32 fine-level fields)
bool mg_available(of_grid* g);
void mg_vcycle(of_grid* g, const float* r, float* z, const double* done);
// z = one V-cycle of (-L_h + sigma) applied to r, sigma > 0 (real fields)
void mg_vcycle_real_shifted(of_grid* g, const float* r, float* z, const double* done, double sigma);
// the same for complex fields and A = -L + sigma (sigma > 0), real and imaginary parts alike
void mg_vcycle_shifted(of_grid* g, const float2* r, float2* z, const double* done, double sigma);

// ion terms (of_atoms.cu)
void pseudocharge(of_grid* g, const of_system* sys, double* b, double* e_self);
void overlap_correction(of_grid* g, const of_system* sys, double* e_c, double* fc_host);
void forces(of_grid* g, const of_system* sys, const double* phi, double* F);

}  // namespace of
