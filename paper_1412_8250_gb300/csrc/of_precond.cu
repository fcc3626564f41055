// Learned preconditioner for the Poisson CG.
//
// Network: three periodic 3x3x3 convolutions, 1 -> 16 -> 16 -> 1 channels with biases, exact
// (erf) GELU after the first two; weights and stored activations in BF16, every sum in FP32.
// The forward pass runs on the tensor cores (tcgen05.mma, accumulators in tensor memory); the
// backward pass of training on the CUDA cores.
// Training loss for one residual r (scaled to unit RMS): the A-norm error of the correction
// y = net(r) against the exact correction e = A^{-1} r, up to the constant 1/2 e^T A e,
//     loss = 1/2 y^T A y - y^T r,   A = -L_h,   d loss / d y = A y - r,
// so the residuals that the solver itself produces are the whole training set.  Applied as
// z = s net(r / s), s the RMS of r, inside a flexible CG that keeps the network's direction
// only while it is a clear descent direction (cos(r, z) > theta) and otherwise takes the plain
// one for that step (Jacobi: the diagonal of A is a constant).  The solve runs as the FP32
// inner solver of the FP64 iterative refinement, whose stopping test is the true FP64
// residual, so the network never sets the answer.  The paper asks for better preconditioning
// of its Krylov solves (Sec. 5.5) without naming one; the plain CG it replaces is Sec. 4's.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "of_krylov.cuh"

struct of_precond {
    float* params = nullptr;      // device FP32 master parameters [NPAR], then grad, m, v
    __nv_bfloat16* pbf = nullptr; // device BF16 copy used by every kernel
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    int step = 0;                 // Adam step count
    int device = 0;
    // limit of the tensor-core kernels' waits for an MMA completion (of_precond_set_wait_limit)
    unsigned long long wait_ns = 2000000000ull;
    // BF16 weights of the backward pass in the forward layout (k_backward_weights)
    __nv_bfloat16* pbw = nullptr;
    // the network stands in for the inverse of -L_h + shift (0: the Poisson operator)
    double shift = 0.0;
};

namespace of {

constexpr int NC = 16;                       // channels
constexpr int NT = 27;                       // taps (dz, dy, dx) in {-1,0,1}^3, z outermost
constexpr int OW1 = 0, OB1 = OW1 + NC * NT;  // W1[o][t], b1[o]
constexpr int OW2 = OB1 + NC, OB2 = OW2 + NC * NC * NT;   // W2[o][c][t], b2[o]
constexpr int OW3 = OB2 + NC, OB3 = OW3 + NC * NT;        // W3[c][t], b3
constexpr int NPAR = OB3 + 1;                // 7809
constexpr int SC_NET = 110;                  // scalars: 110 sum r^2, 111 RMS, 112/113 loss sums
constexpr int FS_OFF = 200;                  // FCG state (FState) in the grid's scalars
constexpr int FDOTS_OFF = 180;               // sums of the flexible CG / COCG direction choice

// Flexible-CG scalars, next to the inner KState.  Directions are kept A-conjugate to the last
// FCG_M ones (truncated FCG, Notay), held in a ring of FCG_M (p, A p) pairs.
constexpr int FCG_M = 4;
struct FState {
    double mean;            // mean of the network output (removed)
    double use_net;         // this step's direction: 1 network, 0 plain
    double net_steps;
    double plain_steps;
    double cos_last;
    double pad[3];
    double pAp[FCG_M];      // p_j^T A p_j per ring slot
    double c[FCG_M];        // next direction = d - sum_j c_j p_j
};
struct Ring {
    float* p[FCG_M];
    float* Ap[FCG_M];
};
inline FState* fstate(of_grid* g) { return (FState*)(g->s.scalars + FS_OFF); }

// Periodic neighbour offsets of one point: index(x + t) = z[a] + y[b] + x[c], t = 9a + 3b + c
struct Nb {
    long long z[3];
    int y[3], x[3];
    // selects instead of array indexing keep the offsets in registers when t is not constant
    __device__ __forceinline__ long long at(int t) const {
        const int a = t / 9, b = (t / 3) % 3, c = t % 3;
        const long long zo = a == 0 ? z[0] : (a == 1 ? z[1] : z[2]);
        const int yo = b == 0 ? y[0] : (b == 1 ? y[1] : y[2]);
        const int xo = c == 0 ? x[0] : (c == 1 ? x[1] : x[2]);
        return zo + yo + xo;
    }
};
__device__ __forceinline__ Nb neighbours(const Dims& d, long long i) {
    const long long plane = (long long)d.n1 * d.n2;
    const int z = (int)(i / plane);
    const int rem = (int)(i - (long long)z * plane);
    const int y = rem / d.n1, x = rem - y * d.n1;
    Nb b;
    b.z[0] = (long long)(z == 0 ? d.n3 - 1 : z - 1) * plane;
    b.z[1] = (long long)z * plane;
    b.z[2] = (long long)(z + 1 == d.n3 ? 0 : z + 1) * plane;
    b.y[0] = (y == 0 ? d.n2 - 1 : y - 1) * d.n1;
    b.y[1] = y * d.n1;
    b.y[2] = (y + 1 == d.n2 ? 0 : y + 1) * d.n1;
    b.x[0] = x == 0 ? d.n1 - 1 : x - 1;
    b.x[1] = x;
    b.x[2] = x + 1 == d.n1 ? 0 : x + 1;
    return b;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void store8(__nv_bfloat16* p, const float (&v)[8]) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    *reinterpret_cast<uint4*>(p) = u;
}

// ---------------------------------------------------------------- forward
// ---------------------------------------------------------------- forward on the tensor cores
// Layer 2 is the network's dense contraction: per point z2[o] = b2[o] + sum_t sum_c
// W2[o][c][t] a1[x+t][c], 432 multiply-adds per output channel.  Over a tile of up to 128
// consecutive points of one x-row it is the implicit GEMM D[128 x 16] = sum_t A_t B_t^T,
// A_t[m][c] = a1[x_m + t][c], B_t[o][c] = W2[o][c][t]: 27 tcgen05.mma of shape M=128, N=16,
// K=16 (BF16 operands, FP32 accumulators in tensor memory), issued by one thread.  The three
// taps dx = -1, 0, 1 of one (dz, dy) plane read the same staged rows shifted by one row, so a
// tile stages nine plane rows of length L + 2 (x0 - 1 .. x0 + L, wrapped) and each MMA's A
// descriptor starts dx + 1 rows into its plane.  Each plane accumulates into its own 16
// columns (nine short chains instead of one of 27).  Layer 3 (one output channel) is the same
// contraction with B_t row 0 = W3[.][t] and rows 1-15 zero.  The epilogue reads the
// accumulators with tcgen05.ld and sums them: layer 2 adds b2, applies GELU and stores BF16
// (z2 too when training); layer 3 takes column 0, adds b3 and scales.  Layer 1 (one input
// channel) is one GEMM with the 27 taps as K, padded to 32.
// Shared-memory operands are K-major without swizzle: core matrices of 8 rows x 16 bytes
// (8 BF16 channels), rows 16 bytes apart throughout (stride byte offset 128 per 8-row group),
// channels 8-15 one plane-half further (leading byte offset = ROWS * 16).
namespace tc {
constexpr int M = 128;                   // rows per MMA (points per tile, padded)
constexpr int THREADS = 256;             // two threads per row: channel halves
constexpr int ROWS = M + 2;              // staged rows per plane: x0 - 1 .. x0 + 128
constexpr int HALF = ROWS * 16;          // bytes of one channel half of a plane (2080)
constexpr int PLANE = 2 * HALF;          // 4160
constexpr int A_BYTES = 9 * PLANE;       // 37440
constexpr int B_TAP = NC * NC * 2;       // 512 bytes per tap: 16 x 16 BF16
constexpr int B_BYTES = NT * B_TAP;      // 13824
constexpr int SMEM = 128 + 2 * A_BYTES + B_BYTES + 64;   // layers 2 and 3: two A buffers
constexpr int SMEM1 = 128 + A_BYTES + 2 * B_TAP + 64;      // layer 1
constexpr int ACC_COLS = 256;   // layers 2 and 3: nine 16-column accumulators (144 used); two
                                // CTAs per SM fill the 512 columns of tensor memory
// layer 1: A tile 128 rows x 32 taps, four K-blocks of 8 taps (2048 bytes each), then the
// staged FP32 planes of r
constexpr int L1_KB = M * 16;
constexpr int L1_STAGE = 4 * L1_KB;
static_assert(L1_STAGE + 9 * ROWS * 4 <= A_BYTES, "layer-1 staging must fit the A buffer");
constexpr uint32_t A_LBO = HALF, A_SBO = 128;    // B tiles: (o/8, c/8) at (o/8)*256 + (c/8)*128
constexpr uint32_t B_LBO = 128, B_SBO = 256;
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NC >> 3) << 17) |
                           ((uint32_t)(M >> 4) << 24);
constexpr unsigned long long WAIT_NS = 2000000000ull;   // give up on a completion after 2 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
// descriptor version 1 (bit 46), no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the phase of parity `parity` of an mbarrier: false once limit_ns have passed
// (at once for limit_ns = 0, without polling)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
    if (limit_ns == 0) return false;
    const unsigned long long t0 = now_ns();
    for (int k = 0; k < (1 << 22); ++k) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((k & 63) == 63 && now_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
// loads without the wait: issue several, then one wait_ld()
__device__ __forceinline__ void ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr) : "memory");
}
__device__ __forceinline__ void ld1_nowait(uint32_t taddr, uint32_t& r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
}  // namespace tc

// Activations a1, a2, z1, z2 are stored channel-half planar: channel c of point i at
// p[((c / 8) * n + i) * 8 + c % 8], so that any run of consecutive points of one half is a
// contiguous block that a bulk copy moves straight into the MMA operand layout.
__device__ __forceinline__ void load16p(const __nv_bfloat16* p, long long n, long long i, float (&v)[NC]) {
    const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(p + i * 8));
    const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(p + (n + i) * 8));
    const __nv_bfloat162* h0 = reinterpret_cast<const __nv_bfloat162*>(&u0);
    const __nv_bfloat162* h1 = reinterpret_cast<const __nv_bfloat162*>(&u1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f0 = __bfloat1622float2(h0[k]);
        const float2 f1 = __bfloat1622float2(h1[k]);
        v[2 * k] = f0.x; v[2 * k + 1] = f0.y;
        v[8 + 2 * k] = f1.x; v[8 + 2 * k + 1] = f1.y;
    }
}
__device__ __forceinline__ float getp(const __nv_bfloat16* p, long long n, long long i, int c) {
    return __bfloat162float(p[((long long)(c >> 3) * n + i) * 8 + (c & 7)]);
}

// B tiles (N = 16 output channels o x K = 16), K-major, (o/8, c/8) core matrices at
// (o/8) * 256 + (c/8) * 128: per tap t for layers 2 and 3, per half h of the 32 padded taps
// for layer 1
template <int LAYER>
__device__ __forceinline__ void fill_b(unsigned char* Bs, const __nv_bfloat16* __restrict__ P, float* bias) {
    const int ntiles_b = LAYER == 1 ? 2 : NT;
    for (int k = threadIdx.x; k < ntiles_b * NC * NC; k += blockDim.x) {
        const int t = k / (NC * NC), o = (k / NC) % NC, c = k % NC;
        __nv_bfloat16 w;
        if (LAYER == 1) {
            const int tap = 16 * t + c;
            w = tap < NT ? P[OW1 + o * NT + tap] : __float2bfloat16(0.f);
        } else if (LAYER == 2) {
            w = P[OW2 + (o * NC + c) * NT + t];
        } else {
            w = o == 0 ? P[OW3 + c * NT + t] : __float2bfloat16(0.f);
        }
        *(__nv_bfloat16*)(Bs + t * tc::B_TAP + (o >> 3) * 256 + (c >> 3) * 128 + (o & 7) * 16 + (c & 7) * 2) = w;
    }
    const int tid = threadIdx.x;
    if (tid < NC)
        bias[tid] = LAYER == 1 ? __bfloat162float(P[OB1 + tid])
                  : LAYER == 2 ? __bfloat162float(P[OB2 + tid])
                               : (tid == 0 ? __bfloat162float(P[OB3]) : 0.f);
}

// first point of the x-row of each plane q = 3 (dz + 1) + (dy + 1) around row (y, z)
__device__ __forceinline__ void plane_bases(const Dims& d, int y, int z, long long (&qb)[9]) {
    const long long plane = (long long)d.n1 * d.n2;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int zz = z + q / 3 - 1, yy = y + q % 3 - 1;
        const int zw = zz < 0 ? zz + d.n3 : (zz >= d.n3 ? zz - d.n3 : zz);
        const int yw = yy < 0 ? yy + d.n2 : (yy >= d.n2 ? yy - d.n2 : yy);
        qb[q] = (long long)zw * plane + (long long)yw * d.n1;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
}
// tensor-memory columns (a power of two >= 32), allocated and freed by one whole warp
template <int COLS>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(tc::smem_addr(slot)), "n"(COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int COLS>
__device__ __forceinline__ void tmem_free(uint32_t tmem) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(COLS) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

// Copies the nine plane rows of a tile (staged row j = point x0 - 1 + j of its x-row, wrapped;
// both channel halves) into an A buffer with 16-byte asynchronous copies, all threads: thread
// tid takes half h = tid / 128 of staged row j = tid % 128 (and of row 128 + j for j < 2) of
// every plane.  With the planar activation layout consecutive threads copy consecutive 16
// bytes, so every 32-byte sector read is used whole.  Commits one copy group.
__device__ __forceinline__ void stage_planes(uint32_t abuf, const __nv_bfloat16* in, long long n,
                                             const long long (&qb)[9], int x0, int L, int n1) {
    const int h = threadIdx.x >> 7;
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int j = (threadIdx.x & (tc::M - 1)) + rep * tc::M;
        if (j < L + 2) {
            int x = x0 - 1 + j;
            x = x < 0 ? x + n1 : (x >= n1 ? x - n1 : x);
            const __nv_bfloat16* src = in + ((long long)h * n + x) * 8;
            const uint32_t dst = abuf + h * tc::HALF + j * 16;
#pragma unroll
            for (int q = 0; q < 9; ++q)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             :: "r"(dst + q * tc::PLANE), "l"(src + qb[q] * 8) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Layer 1: z1 = W1 * (sgn r / s) + b1, a1 = GELU(z1), as the GEMM D[128 x 16] = A B^T with
// Data-gradient epilogue (the backward pass runs the forward kernels with the mirrored,
// transposed weights of of_precond's backward array): the convolution's 8 channels ch*8 ..
// of point i times GELU' of the forward pre-activation zin, to gout (FP32, [x][16], for the
// weight gradients) and, when aout is set, to aout (BF16 planar, the next convolution's input).
__device__ __forceinline__ void epilogue_bwd(const float (&acc)[8], const __nv_bfloat16* zin, float* gout,
                                             __nv_bfloat16* aout, long long n, long long i, int ch) {
    float z[8];
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(zin + ((long long)ch * n + i) * 8));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        z[2 * k] = f.x;
        z[2 * k + 1] = f.y;
    }
    float g[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) g[o] = acc[o] * gelu_grad_f(z[o]);
    float4* go = reinterpret_cast<float4*>(gout + i * NC + 8 * ch);
    go[0] = make_float4(g[0], g[1], g[2], g[3]);
    go[1] = make_float4(g[4], g[5], g[6], g[7]);
    if (aout) store8(aout + ((long long)ch * n + i) * 8, g);
}

// A[m][k] = (sgn r / s)(x_m + t_k) (taps k < 27, zero up to 32) and B[o][k] = W1[o][t_k]: two
// MMAs of K = 16.  The nine plane rows of r are staged in FP32 (plain loads), each thread
// builds half of its A row in BF16.  rnout: the input as rounded to BF16 (training).  One CTA
// of 256 threads per tile; thread tid owns row m = tid % 128 and channels 8 (tid / 128) .. + 7.
template <bool BWD>
__global__ void __launch_bounds__(tc::THREADS, 4) k_conv1_tc(Dims d, int nseg, int lseg,
                                                             const float* __restrict__ rin,
                                                             const __nv_bfloat16* __restrict__ P,
                                                             __nv_bfloat16* zout, __nv_bfloat16* aout,
                                                             float* rnout, const double* s_dev, float sgn,
                                                             double* err, unsigned long long wait_ns,
                                                             const __nv_bfloat16* __restrict__ zin,
                                                             float* gout) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned char* As = sm;
    unsigned char* Bs = sm + tc::A_BYTES;
    uint64_t* bar = (uint64_t*)(Bs + 2 * tc::B_TAP);
    uint32_t* tslot = (uint32_t*)(bar + 1);
    __shared__ float bias[NC];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (tc::M - 1), ch = tid >> 7;
    for (int k = tid; k < tc::A_BYTES / 16; k += tc::THREADS)
        reinterpret_cast<uint4*>(As)[k] = make_uint4(0, 0, 0, 0);
    fill_b<1>(Bs, P, bias);
    const uint32_t bar_a = tc::smem_addr(bar);
    if (tid == 0) {
        mbar_init(bar_a);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc<32>(tslot);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t a_base = tc::smem_addr(As), b_base = tc::smem_addr(Bs);
    // the input scaled by sgn / RMS (forward), or as it is (data gradient)
    const double rms = BWD ? 1.0 : *s_dev;
    const float inv = rms > 0.0 ? sgn * (float)(1.0 / rms) : 0.f;   // 0 for a zero residual
    const long long ntiles = (long long)d.n2 * d.n3 * nseg;
    float* rs = reinterpret_cast<float*>(As + tc::L1_STAGE);
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = (int)blockIdx.x; ok && tile < ntiles; tile += (int)gridDim.x) {
        const int rowi = tile / nseg;
        const int x0 = (tile - rowi * nseg) * lseg;
        const int L = min(lseg, d.n1 - x0);
        const int z = rowi / d.n2;
        long long qb[9];
        plane_bases(d, rowi - z * d.n2, z, qb);
        if (tid < L + 2) {   // staged row j = tid, point x0 - 1 + j (wrapped)
            int x = x0 - 1 + tid;
            x = x < 0 ? x + d.n1 : (x >= d.n1 ? x - d.n1 : x);
            float v[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = __ldg(rin + qb[q] + x);
#pragma unroll
            for (int q = 0; q < 9; ++q) rs[q * tc::ROWS + tid] = v[q] * inv;
        }
        __syncthreads();
        __nv_bfloat16 row[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int t = 16 * ch + u;
            row[u] = __float2bfloat16(t < NT ? rs[(t / 3) * tc::ROWS + m + t % 3] : 0.f);
        }
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
            *(uint4*)(As + (2 * ch + kb) * tc::L1_KB + m * 16) = *reinterpret_cast<const uint4*>(row + 8 * kb);
        if (rnout && ch == 0 && m < L)   // tap 13 is the point itself
            rnout[(long long)rowi * d.n1 + x0 + m] = __bfloat162float(row[13]);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h)
                tc::mma(tmem, tc::desc(a_base + 2 * h * tc::L1_KB, tc::L1_KB, tc::A_SBO),
                        tc::desc(b_base + h * tc::B_TAP, tc::B_LBO, tc::B_SBO), h > 0 ? 1u : 0u);
            mma_commit(bar_a);
        }
        const bool seen = tc::mbar_wait(bar_a, phase, wait_ns);
        phase ^= 1u;
        ok = __syncthreads_and(seen) != 0;
        tc::fence_after();
        if (!ok) break;
        float acc[8];
        tc::ld8(tmem + ((uint32_t)((warp & 3) * 32) << 16) + 8 * ch, acc);
        if (m < L) {
            const long long i = (long long)rowi * d.n1 + x0 + m;
            if (BWD)
                epilogue_bwd(acc, zin, gout, aout, d.n, i, ch);
            else {
                float zv[8], g[8];
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    zv[o] = acc[o] + bias[8 * ch + o];
                    g[o] = gelu_f(zv[o]);
                }
                if (zout) store8(zout + ((long long)ch * d.n + i) * 8, zv);
                store8(aout + ((long long)ch * d.n + i) * 8, g);
            }
        }
        tc::fence_before();
    }
    if (!ok) {
        if (tid == 0) *err = 1.0;
        // let the MMAs still in flight finish (bounded by the full limit, whatever wait_ns was)
        // before the tensor memory they write is freed
        tc::mbar_wait(bar_a, phase ^ 1u, tc::WAIT_NS);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tmem_free<32>(tmem);
}

// Layers 2 and 3 (see above).  LAYER 2: in = a1 -> z2 (optional), a2.  LAYER 3: in = a2 ->
// y = scale (W3 * a2 + b3), scale = *s_dev (1 with s_dev null).  The next tile's plane rows are
// copied into the other A buffer while the current tile's MMAs and epilogue run; one CTA of 256
// threads per tile, persistent; err as for layer 1.
template <int LAYER, bool BWD>
__global__ void __launch_bounds__(tc::THREADS, 2) k_conv_tc(Dims d, int nseg, int lseg,
                                                            const __nv_bfloat16* __restrict__ in,
                                                            const __nv_bfloat16* __restrict__ P,
                                                            __nv_bfloat16* zout, __nv_bfloat16* aout,
                                                            float* yout, const double* s_dev, double* err,
                                                            unsigned long long wait_ns,
                                                            const __nv_bfloat16* __restrict__ zin,
                                                            float* gout) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned char* As = sm;                              // two A buffers
    unsigned char* Bs = sm + 2 * tc::A_BYTES;
    uint64_t* bar = (uint64_t*)(Bs + tc::B_BYTES);       // MMA completion
    uint32_t* tslot = (uint32_t*)(bar + 1);
    __shared__ float bias[NC];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (tc::M - 1), ch = tid >> 7;
    for (int k = tid; k < 2 * tc::A_BYTES / 16; k += tc::THREADS)   // finite values in unused rows
        reinterpret_cast<uint4*>(As)[k] = make_uint4(0, 0, 0, 0);
    fill_b<LAYER>(Bs, P, bias);
    const uint32_t bar_m = tc::smem_addr(bar);
    if (tid == 0) {
        mbar_init(bar_m);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc<tc::ACC_COLS>(tslot);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t a_base = tc::smem_addr(As), b_base = tc::smem_addr(Bs);
    const float scale = (LAYER == 3 && s_dev) ? (float)*s_dev : 1.f;
    const long long ntiles = (long long)d.n2 * d.n3 * nseg;
    // tile -> x-row rowi = y + n2 z, segment start x0, length L (32-bit: the host keeps the
    // tile count below 2^31)
    auto geom = [&](int tile, int& rowi, int& x0, int& L) {
        rowi = tile / nseg;
        x0 = (tile - rowi * nseg) * lseg;
        L = min(lseg, d.n1 - x0);
    };
    auto stage = [&](int tile, int b) {
        int rowi, x0, L;
        geom(tile, rowi, x0, L);
        const int z = rowi / d.n2;
        long long qb[9];
        plane_bases(d, rowi - z * d.n2, z, qb);
        stage_planes(a_base + b * tc::A_BYTES, in, d.n, qb, x0, L, d.n1);
    };
    if ((long long)blockIdx.x < ntiles) stage((int)blockIdx.x, 0);
    uint32_t phase = 0;
    bool ok = true;
    int k = 0;
    for (int tile = (int)blockIdx.x; tile < ntiles; tile += (int)gridDim.x, ++k) {
        const int b = k & 1;
        const long long next = (long long)tile + gridDim.x;
        if (next < ntiles) {   // the other buffer's MMAs completed in the previous iteration
            stage((int)next, b ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t abuf = a_base + b * tc::A_BYTES;
            // tap t reads plane q = t / 3 shifted dx + 1 = t % 3 rows and accumulates into
            // accumulator q (columns 16 q ..): nine independent chains of three MMAs, issued
            // dx-major so that consecutive MMAs never share an accumulator
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int t = 3 * q + dx;
                    tc::mma(tmem + NC * q, tc::desc(abuf + q * tc::PLANE + dx * 16, tc::A_LBO, tc::A_SBO),
                            tc::desc(b_base + t * tc::B_TAP, tc::B_LBO, tc::B_SBO), dx > 0 ? 1u : 0u);
                }
            mma_commit(bar_m);
        }
        const bool done = tc::mbar_wait(bar_m, phase, wait_ns);
        ok = __syncthreads_and(done) != 0;
        tc::fence_after();
        if (!ok) break;
        phase ^= 1u;
        int rowi, x0, L;
        geom(tile, rowi, x0, L);
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const long long i = (long long)rowi * d.n1 + x0 + m;
        if (LAYER == 2) {
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            uint32_t part[9][8];   // the nine plane accumulators, loaded together
#pragma unroll
            for (int q = 0; q < 9; ++q) tc::ld8_nowait(taddr + NC * q + 8 * ch, part[q]);
            tc::wait_ld();
#pragma unroll
            for (int q = 0; q < 9; ++q)
#pragma unroll
                for (int o = 0; o < 8; ++o) acc[o] += __uint_as_float(part[q][o]);
            if (m < L) {
                if (BWD)
                    epilogue_bwd(acc, zin, gout, aout, d.n, i, ch);
                else {
                    float zv[8], g[8];
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        zv[o] = acc[o] + bias[8 * ch + o];
                        g[o] = gelu_f(zv[o]);
                    }
                    if (zout) store8(zout + ((long long)ch * d.n + i) * 8, zv);
                    store8(aout + ((long long)ch * d.n + i) * 8, g);
                }
            }
        } else if (ch == 0) {
            uint32_t part[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) tc::ld1_nowait(taddr + NC * q, part[q]);
            tc::wait_ld();
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) v += __uint_as_float(part[q]);
            if (m < L) yout[i] = scale * (v + bias[0]);
        }
        tc::fence_before();   // the next tile's MMAs overwrite the accumulators
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the CTA
    if (!ok) {
        if (tid == 0) *err = 1.0;
        // let the MMAs still in flight finish (bounded by the full limit, whatever wait_ns was)
        // before the tensor memory they write is freed
        tc::mbar_wait(bar_m, phase, tc::WAIT_NS);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tmem_free<tc::ACC_COLS>(tmem);
}

// ---------------------------------------------------------------- backward
// The data gradients run on the tensor-core kernels above (k_backward_weights); the weight
// and bias gradients here, on the CUDA cores in FP32.
// Weight and bias gradients.  A persistent grid walks tiles of WT consecutive points; per
// tile and tap t the shifted activations a1(x+t), a2(x+t), rn(x+t) are gathered into shared
// memory, and
//   thread (o, c) of 256:          dW2[o][c][t] += sum_x gz2[x][o] a1[x+t][c]
//   warp 0, lanes 0-15 (c):        dW3[c][t]    += sum_x gy[x] a2[x+t][c]
//   warp 0, lanes 16-31 (o):       dW1[o][t]    += sum_x gz1[x][o] rn[x+t]
// with the biases summed once per tile.  Each block writes its FP32 sums to part[block][*];
// k_sum_parts adds the blocks in a fixed order.
constexpr int WT = 128;
__global__ void __launch_bounds__(256) k_net_wgrad(Dims d, const float* __restrict__ rn,
                                                   const __nv_bfloat16* __restrict__ a1,
                                                   const __nv_bfloat16* __restrict__ a2,
                                                   const float* __restrict__ gz1,
                                                   const float* __restrict__ gz2,
                                                   const float* __restrict__ gy, float* part) {
    __shared__ float s_g2[WT][NC + 1];
    __shared__ float s_g1[WT][NC + 1];
    __shared__ float s_a1[WT][NC + 1];
    __shared__ float s_a2[WT][NC + 1];
    __shared__ float s_gy[WT];
    __shared__ float s_rn[WT];
    __shared__ long long s_idx[WT];
    const int tid = threadIdx.x;
    const int o2 = tid / NC, c2 = tid % NC;
    const int lane = tid & 31;
    const bool w0 = tid < 32;
    float acc2[NT], accx[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc2[t] = accx[t] = 0.f;
    float accb2 = 0.f, accbx = 0.f;
    const long long ntiles = (d.n + WT - 1) / WT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long x0 = tile * WT;
        __syncthreads();
        for (int k = tid; k < WT * NC; k += blockDim.x) {
            const int p = k / NC, c = k % NC;
            const long long x = x0 + p;
            const bool in = x < d.n;
            s_g2[p][c] = in ? gz2[x * NC + c] : 0.f;
            s_g1[p][c] = in ? gz1[x * NC + c] : 0.f;
        }
        for (int p = tid; p < WT; p += blockDim.x) s_gy[p] = (x0 + p < d.n) ? gy[x0 + p] : 0.f;
        __syncthreads();
        if (c2 == 0)
            for (int p = 0; p < WT; ++p) accb2 += s_g2[p][o2];
        if (w0 && lane < NC)
            for (int p = 0; p < WT; ++p) accbx += s_g1[p][lane];
        else if (w0 && lane == NC)
            for (int p = 0; p < WT; ++p) accbx += s_gy[p];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            __syncthreads();
            for (int p = tid; p < WT; p += blockDim.x) {
                const long long x = x0 + p;
                s_idx[p] = x < d.n ? neighbours(d, x).at(t) : -1;
            }
            __syncthreads();
            for (int k = tid; k < WT * NC; k += blockDim.x) {
                const int p = k / NC, c = k % NC;
                const long long j = s_idx[p];
                s_a1[p][c] = j >= 0 ? getp(a1, d.n, j, c) : 0.f;
                s_a2[p][c] = j >= 0 ? getp(a2, d.n, j, c) : 0.f;
            }
            for (int p = tid; p < WT; p += blockDim.x) s_rn[p] = s_idx[p] >= 0 ? rn[s_idx[p]] : 0.f;
            __syncthreads();
            float s = 0.f;
#pragma unroll 8
            for (int p = 0; p < WT; ++p) s = fmaf(s_g2[p][o2], s_a1[p][c2], s);
            acc2[t] += s;
            if (w0) {
                float sx = 0.f;
                if (lane < NC) {
#pragma unroll 8
                    for (int p = 0; p < WT; ++p) sx = fmaf(s_gy[p], s_a2[p][lane], sx);
                } else {
#pragma unroll 8
                    for (int p = 0; p < WT; ++p) sx = fmaf(s_g1[p][lane - NC], s_rn[p], sx);
                }
                accx[t] += sx;
            }
        }
    }
    float* out = part + (long long)blockIdx.x * NPAR;
#pragma unroll
    for (int t = 0; t < NT; ++t) out[OW2 + (o2 * NC + c2) * NT + t] = acc2[t];
    if (c2 == 0) out[OB2 + o2] = accb2;
    if (w0) {
        if (lane < NC) {
#pragma unroll
            for (int t = 0; t < NT; ++t) out[OW3 + lane * NT + t] = accx[t];
            out[OB1 + lane] = accbx;
        } else {
#pragma unroll
            for (int t = 0; t < NT; ++t) out[OW1 + (lane - NC) * NT + t] = accx[t];
            if (lane == NC) out[OB3] = accbx;
        }
    }
}

__global__ void k_sum_parts(int nblocks, const float* __restrict__ part, float* grad, float scale) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(long long)b * NPAR + p];
    grad[p] += scale * s;
}

// loss sums y^T A y and y^T rn into out[0], out[1]; gy = A y - rn
__global__ void __launch_bounds__(256) k_net_loss(long long n, const float* __restrict__ y,
                                                  const float* __restrict__ Ay,
                                                  const float* __restrict__ rn, float* gy, RedCtx rc) {
    float p0 = 0.f, p1 = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = Ay[i], yy = y[i], r = rn[i];
        p0 += yy * a;
        p1 += yy * r;
        gy[i] = a - r;
    }
    double acc[2] = {(double)p0, (double)p1};
    grid_reduce<2>(acc, rc.partials, rc.counter, rc.out);
}

// out[0] = sum x^2, out[1] = RMS of x
__global__ void __launch_bounds__(256) k_rms32(long long n, const float* __restrict__ x, RedCtx rc) {
    float p = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p = fmaf(x[i], x[i], p);
    double acc[1] = {(double)p};
    if (grid_reduce<1>(acc, rc.partials, rc.counter, rc.out) && threadIdx.x == 0)
        rc.out[1] = sqrt(acc[0] / (double)n);
}

// Adam (Kingma & Ba) with bias correction; refreshes the BF16 copy and clears the gradient
__global__ void k_adam(float* params, __nv_bfloat16* pbf, float* grad, float* m, float* v, float lr,
                       float b1, float b2, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float w = params[p] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
    params[p] = w;
    pbf[p] = __float2bfloat16(w);
    grad[p] = 0.f;
}

// The data gradients of layers 3 and 2 are convolutions of the same shape as layers 1 and 2:
//   ga2[c](x) = sum_t W3[c][t] gy(x - t) = sum_t' W3[c][mirror t'] gy(x + t')        (1 -> 16)
//   ga1[c](x) = sum_o sum_t W2[o][c][t] gz2[o](x - t) = sum_t' sum_o W2[o][c][mirror t'] gz2[o](x + t')
// so they run on the forward tensor-core kernels with W1' = mirrored W3 and W2' = W2 with its
// channels transposed and taps mirrored (mirror t = NT - 1 - t negates the offset), zero biases.
__global__ void k_backward_weights(const __nv_bfloat16* __restrict__ P, __nv_bfloat16* __restrict__ Q) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPAR) return;
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (k >= OW1 && k < OB1) {
        const int c = (k - OW1) / NT, t = (k - OW1) % NT;
        v = P[OW3 + c * NT + (NT - 1 - t)];
    } else if (k >= OW2 && k < OB2) {
        const int j = k - OW2, cc = j / (NC * NT), o = (j / NT) % NC, t = j % NT;
        v = P[OW2 + (o * NC + cc) * NT + (NT - 1 - t)];
    }
    Q[k] = v;
}

__global__ void k_to_bf16(int n, const float* a, __nv_bfloat16* b) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) b[p] = __float2bfloat16(a[p]);
}

// ---------------------------------------------------------------- flexible CG kernels
// Ap = A p (A = -L) into ring slot `slot`; reduces p^T A p and r^T p, sets alpha
struct OpFcgA {
    static constexpr int kClass = PC_CG_F32, kWords = 3;
    const float* p;
    const float* r;
    float* Ap;
    KState* st;
    FState* fs;
    int slot;
    RedCtx rc;
    float shift;   // A = -L_h + shift
    float acc[2];
    __device__ bool begin() {
        if (st->done != 0.0) return false;
        acc[0] = acc[1] = 0.f;
        return true;
    }
    __device__ float load(long long i) const { return p[i]; }
    __device__ float2 load2(long long i) const { return *reinterpret_cast<const float2*>(p + i); }
    __device__ void store(long long i, float c, float lap) {
        const float q = fmaf(shift, c, -lap);
        Ap[i] = q;
        acc[0] = fmaf(c, q, acc[0]);
        acc[1] = fmaf(r[i], c, acc[1]);
    }
    __device__ void end() {
        double a[2] = {(double)acc[0], (double)acc[1]};
        if (grid_reduce<2>(a, rc.partials, rc.counter, st->red) && threadIdx.x == 0 && threadIdx.y == 0) {
            st->pAp_re = a[0];
            fs->pAp[slot] = a[0];
            if (!(a[0] > 0.0)) {
                st->breakdown = 1.0;
                st->done = 1.0;
            } else {
                st->alpha_re = a[1] / a[0];
            }
        }
    }
};

// x += alpha p ; r_new = r - alpha A p ; |r_new|^2, iteration count, stop flag
__global__ void __launch_bounds__(256) k_fcg_update(long long n, float* __restrict__ x,
                                                    const float* __restrict__ r, float* __restrict__ rnew,
                                                    const float* __restrict__ p,
                                                    const float* __restrict__ Ap, KState* st, RedCtx rc) {
    if (st->done != 0.0) return;
    const float al = (float)st->alpha_re;
    float part = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] = fmaf(al, p[i], x[i]);
        const float v = fmaf(-al, Ap[i], r[i]);
        rnew[i] = v;
        part = fmaf(v, v, part);
    }
    double acc[1] = {(double)part};
    if (grid_reduce<1>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->rr = acc[0];
        st->iters += 1.0;
        if (acc[0] <= st->tol2 || st->iters >= st->maxit) st->done = 1.0;
    }
}

// Sums for the choice of the next direction: sum z, sum r, r.z, z.z and, per filled ring slot
// j < valid, z.Ap_j and r.Ap_j.  The last block keeps the network direction d = z - mean(z)
// (project: the Poisson operator, whose null space is the constants; else d = z) when
// cos(r, d) > theta, else d = r, and sets c_j = d.Ap_j / p_j.Ap_j (sum Ap_j = 0 for the
// Laplacian, so the mean shift drops out of d.Ap_j).
constexpr int DOTS_K = 4 + 2 * FCG_M;
static_assert(KS32 + KSTATE_DOUBLES <= FDOTS_OFF && FDOTS_OFF + DOTS_K <= FS_OFF,
              "scalar slots of the flexible-CG sums");
__global__ void __launch_bounds__(256) k_fcg_dots(long long n, const float* __restrict__ r,
                                                  const float* __restrict__ z, int has_net, int project,
                                                  double theta, Ring ring, int valid, KState* st,
                                                  FState* fs, RedCtx rc) {
    if (st->done != 0.0) return;
    float s[DOTS_K];
#pragma unroll
    for (int k = 0; k < DOTS_K; ++k) s[k] = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float rv = r[i];
        const float zv = has_net ? z[i] : rv;
        s[0] += zv;
        s[1] += rv;
        s[2] = fmaf(rv, zv, s[2]);
        s[3] = fmaf(zv, zv, s[3]);
#pragma unroll
        for (int j = 0; j < FCG_M; ++j)
            if (j < valid) {
                const float a = ring.Ap[j][i];
                s[4 + 2 * j] = fmaf(zv, a, s[4 + 2 * j]);
                s[5 + 2 * j] = fmaf(rv, a, s[5 + 2 * j]);
            }
    }
    double acc[DOTS_K];
#pragma unroll
    for (int k = 0; k < DOTS_K; ++k) acc[k] = (double)s[k];
    if (grid_reduce<DOTS_K>(acc, rc.partials, rc.counter, rc.out) && threadIdx.x == 0) {
        const double rr = st->rr;
        bool use = false;
        double mean = 0.0;
        if (has_net) {
            mean = project ? acc[0] / (double)n : 0.0;
            const double zz = acc[3] - (double)n * mean * mean;
            const double rzn = acc[2] - mean * acc[1];
            const double c = (zz > 0.0 && rr > 0.0) ? rzn / sqrt(zz * rr) : -1.0;
            fs->cos_last = c;
            use = c > theta;
        }
        for (int j = 0; j < FCG_M; ++j) {
            const double dA = use ? acc[4 + 2 * j] : acc[5 + 2 * j];
            fs->c[j] = (j < valid && fs->pAp[j] > 0.0) ? dA / fs->pAp[j] : 0.0;
        }
        fs->mean = use ? mean : 0.0;
        fs->use_net = use ? 1.0 : 0.0;
        if (use) fs->net_steps += 1.0; else fs->plain_steps += 1.0;
    }
}

// out = d - sum_{j < valid} c_j p_j,  d = network ? z - mean : r.  out may be the oldest ring
// slot: each element is read before it is written, by the same thread.
__global__ void __launch_bounds__(256) k_fcg_direction(long long n, const float* __restrict__ r,
                                                       const float* __restrict__ z, Ring ring, int valid,
                                                       float* out, const KState* st, const FState* fs) {
    if (st->done != 0.0) return;
    const bool use = fs->use_net != 0.0;
    const float mean = (float)fs->mean;
    float c[FCG_M];
#pragma unroll
    for (int j = 0; j < FCG_M; ++j) c[j] = (float)fs->c[j];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = use ? z[i] - mean : r[i];
#pragma unroll
        for (int j = 0; j < FCG_M; ++j)
            if (j < valid) v = fmaf(-c[j], ring.p[j][i], v);
        out[i] = v;
    }
}

__global__ void k_fcg_reset(FState* fs) {
    fs->mean = 0.0;
    fs->use_net = 0.0;
    fs->net_steps = 0.0;
    fs->plain_steps = 0.0;
    fs->cos_last = 0.0;
    for (int j = 0; j < FCG_M; ++j) fs->pAp[j] = fs->c[j] = 0.0;
}

// ---------------------------------------------------------------- flexible GMRES
// The shifted kernel systems a (-L_h) x + Q x = b are complex symmetric, not Hermitian.  The
// network is trained for the real positive operator A_r = -L_h + c, c = |Q| / a, whose inverse
// applied to the real and imaginary parts separately is a good preconditioner of them (the
// multigrid path uses a V-cycle of the same operator).  Applied directly, the network is not
// accurate enough (flexible COCG and flexible GMRES with z = net(v) stagnated): it is used
// where flexible CG is robust, in a few flexible-CG steps on A_r z = v (to GM_TAU), and those
// inner solves precondition flexible GMRES(GM_M), which keeps every preconditioned vector of a
// cycle and takes the iterate of least residual over their span: Arnoldi with classical
// Gram-Schmidt applied twice (each pass one grid reduction of all projections), the small
// Hessenberg least-squares problem by Givens rotations on the host.
constexpr int GM_M = 8;                        // restart length
constexpr double GM_TAU = 0.1;                 // relative residual of the inner solves
constexpr int GM_INNER_MAX = 40;               // iterations of one inner solve, at most
constexpr int GH1 = FS_OFF + (int)(sizeof(FState) / sizeof(double));   // projections, first pass
constexpr int GH2 = GH1 + 2 * GM_M;            // second pass
constexpr int GNRM = GH2 + 2 * GM_M;           // |w|^2 after orthogonalisation, or |r|^2
static_assert(GNRM + 1 <= KS_NEST, "grid scalars");

struct VecSet {
    float2* v[GM_M + 1];
};
struct GmCoef {
    double2 y[GM_M];
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// out[2k], out[2k+1] = sum_i conj(v_k[i]) w[i] for k < nv, 0 beyond
__global__ void __launch_bounds__(256) k_gm_dots(long long n, const float2* __restrict__ w, VecSet V,
                                                 int nv, RedCtx rc) {
    float s[2 * GM_M];
#pragma unroll
    for (int k = 0; k < 2 * GM_M; ++k) s[k] = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 wv = w[i];
#pragma unroll
        for (int k = 0; k < GM_M; ++k)
            if (k < nv) {
                const float2 v = V.v[k][i];
                s[2 * k] = fmaf(v.x, wv.x, fmaf(v.y, wv.y, s[2 * k]));
                s[2 * k + 1] = fmaf(v.x, wv.y, fmaf(-v.y, wv.x, s[2 * k + 1]));
            }
    }
    double acc[2 * GM_M];
#pragma unroll
    for (int k = 0; k < 2 * GM_M; ++k) acc[k] = (double)s[k];
    grid_reduce<2 * GM_M>(acc, rc.partials, rc.counter, rc.out);
}

// w -= sum_{k < nv} h_k v_k, h_k = (h[2k], h[2k+1]); with norm != 0, |w|^2 into rc.out[0]
__global__ void __launch_bounds__(256) k_gm_orth(long long n, float2* __restrict__ w, VecSet V, int nv,
                                                 const double* __restrict__ h, int norm, RedCtx rc) {
    float2 c[GM_M];
#pragma unroll
    for (int k = 0; k < GM_M; ++k)
        c[k] = k < nv ? make_float2((float)h[2 * k], (float)h[2 * k + 1]) : make_float2(0.f, 0.f);
    float part = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float2 x = w[i];
#pragma unroll
        for (int k = 0; k < GM_M; ++k)
            if (k < nv) {
                const float2 t = cmulf(c[k], V.v[k][i]);
                x.x -= t.x;
                x.y -= t.y;
            }
        w[i] = x;
        part = fmaf(x.x, x.x, fmaf(x.y, x.y, part));
    }
    if (norm) {
        double acc[1] = {(double)part};
        grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
    }
}

// out = s w
__global__ void __launch_bounds__(256) k_gm_scale(long long n, const float2* __restrict__ w,
                                                  float2* __restrict__ out, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = w[i];
        out[i] = make_float2(s * v.x, s * v.y);
    }
}

// real and imaginary parts of v as two planes
__global__ void __launch_bounds__(256) k_split2(long long n, const float2* __restrict__ v, float* __restrict__ rs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 x = v[i];
        rs[i] = x.x;
        rs[n + i] = x.y;
    }
}

// Start of an inner solve of A_r x = r: x = 0, |r|^2 and the stopping state (relative tau)
__global__ void __launch_bounds__(256) k_nest_init(long long n, const float* __restrict__ r,
                                                   float* __restrict__ x, double tau, int maxit,
                                                   KState* st, RedCtx rc) {
    float p = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = r[i];
        x[i] = 0.f;
        p = fmaf(v, v, p);
    }
    double acc[1] = {(double)p};
    if (grid_reduce<1>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->rr = acc[0];
        st->tol2 = tau * tau * acc[0];
        st->done = acc[0] > 0.0 ? 0.0 : 1.0;
        st->iters = 0.0;
        st->maxit = maxit;
        st->breakdown = 0.0;
        st->zshift = 0.0;
    }
}

// out = z[0..n) + i z[n..2n)
__global__ void __launch_bounds__(256) k_merge2(long long n, const float* __restrict__ z, float2* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = make_float2(z[i], z[n + i]);
}

// w = A z, A = a(-L_h) + Q
struct OpGmA {
    static constexpr int kClass = PC_COCG_F32, kWords = 2;
    const float2* z;
    float2* w;
    float a;
    double2 Q;
    __device__ bool begin() { return true; }
    __device__ float2 load(long long i) const { return z[i]; }
    __device__ void store(long long i, float2 c, float2 lap) { w[i] = apply_A(c, lap, a, Q); }
    __device__ void end() {}
};

// r = b - A x and |r|^2 into rc.out[0]
struct OpGmResid {
    static constexpr int kClass = PC_COCG_F32, kWords = 3;
    const float2* x;
    const float2* b;
    float2* r;
    float a;
    double2 Q;
    RedCtx rc;
    float acc;
    __device__ bool begin() {
        acc = 0.f;
        return true;
    }
    __device__ float2 load(long long i) const { return x[i]; }
    __device__ void store(long long i, float2 c, float2 lap) {
        const float2 q = apply_A(c, lap, a, Q), bv = b[i];
        const float2 v = make_float2(bv.x - q.x, bv.y - q.y);
        r[i] = v;
        acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
    }
    __device__ void end() {
        double v[1] = {(double)acc};
        grid_reduce<1>(v, rc.partials, rc.counter, rc.out);
    }
};

// x += sum_{k < m} y_k Z_k
__global__ void __launch_bounds__(256) k_gm_xupdate(long long n, float2* __restrict__ x, VecSet Z, int m,
                                                    GmCoef y) {
    float2 c[GM_M];
#pragma unroll
    for (int k = 0; k < GM_M; ++k) c[k] = make_float2((float)y.y[k].x, (float)y.y[k].y);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float2 v = x[i];
#pragma unroll
        for (int k = 0; k < GM_M; ++k)
            if (k < m) {
                const float2 t = cmulf(c[k], Z.v[k][i]);
                v.x += t.x;
                v.y += t.y;
            }
        x[i] = v;
    }
}

// FP64 right-hand side -> FP32 at unit RMS (sample collection); fresh inner state
__global__ void __launch_bounds__(256) k_unit32(long long n, const double* __restrict__ b, float* r32,
                                                float* e32, const double* sumsq, double tol, int maxit,
                                                KState* st, RedCtx rc) {
    const double ss = *sumsq;
    const double inv = ss > 0.0 ? rsqrt(ss / (double)n) : 1.0;
    float part = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(b[i] * inv);
        r32[i] = v;
        e32[i] = 0.f;
        part = fmaf(v, v, part);
    }
    double acc[1] = {(double)part};
    if (grid_reduce<1>(acc, rc.partials, rc.counter, st->red) && threadIdx.x == 0) {
        st->rr = acc[0];
        st->tol2 = tol * tol * acc[0];
        st->done = (acc[0] <= st->tol2) ? 1.0 : 0.0;
        st->iters = 0.0;
        st->maxit = maxit;
        st->breakdown = 0.0;
        st->scale = 1.0 / inv;
    }
}

__global__ void __launch_bounds__(256) k_sumsq64(long long n, const double* __restrict__ x, RedCtx rc) {
    double p = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p = fma(x[i], x[i], p);
    double acc[1] = {p};
    grid_reduce<1>(acc, rc.partials, rc.counter, rc.out);
}

// ---------------------------------------------------------------- host side
struct NetBufs {
    __nv_bfloat16 *a1, *a2, *z1, *z2, *gz2b;   // gz2b: gz2 in BF16, input of the layer-2 data gradient
    float *y, *Ay, *gy, *rn, *gz2, *gz1, *part;
    int wblocks;
};

static inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

static int wgrad_blocks(long long n) {
    const long long tiles = (n + WT - 1) / WT;
    return (int)std::max(1LL, std::min(tiles, 2LL * num_sms()));
}

// Workspace of the network: the inference part (a1, a2) comes first, so that applying the
// network needs 64 bytes per point and training 272.
static NetBufs net_bufs(of_grid* g, bool training) {
    const size_t n = (size_t)g->d.n;
    const int wb = wgrad_blocks(g->d.n);
    const size_t act = al256(n * NC * sizeof(__nv_bfloat16));
    const size_t f1 = al256(n * sizeof(float)), f16 = al256(n * NC * sizeof(float));
    const size_t bytes = training ? 5 * act + 4 * f1 + 2 * f16 + al256((size_t)wb * NPAR * 4) : 2 * act;
    char* p = (char*)ws(g, WS_K6, bytes);
    NetBufs B{};
    B.a1 = (__nv_bfloat16*)p; p += act;
    B.a2 = (__nv_bfloat16*)p; p += act;
    B.wblocks = wb;
    if (!training) return B;
    B.z1 = (__nv_bfloat16*)p; p += act;
    B.z2 = (__nv_bfloat16*)p; p += act;
    B.gz2b = (__nv_bfloat16*)p; p += act;
    B.y = (float*)p; p += f1;
    B.Ay = (float*)p; p += f1;
    B.gy = (float*)p; p += f1;
    B.rn = (float*)p; p += f1;
    B.gz2 = (float*)p; p += f16;
    B.gz1 = (float*)p; p += f16;
    B.part = (float*)p;
    return B;
}

// y = A x for FP32 fields, A = -L
// y = -L_h x + shift x
struct OpNegLap32 {
    const float* x;
    float* y;
    float shift;
    __device__ bool begin() { return true; }
    __device__ float load(long long i) const { return x[i]; }
    __device__ void store(long long i, float c, float lap) { y[i] = fmaf(shift, c, -lap); }
    __device__ void end() {}
};

constexpr int SC_NET_ERR = SC_NET + 4;   // set by k_net_l2_tc when a wait gave up

static void net_reset_error(of_grid* g) {
    OF_CUDA(cudaMemsetAsync(g->s.scalars + SC_NET_ERR, 0, sizeof(double), g->stream));
}
static void net_check_error(of_grid* g) {
    double e = 0.0;
    fetch_scalars(g, SC_NET_ERR, 1, &e);
    OF_REQUIRE(e == 0.0, OF_ETIMEOUT,
               "tensor-core convolution: an MMA completion was not seen within the wait limit");
}

// The tensor-core layers: x-rows cut into segments of at most 128 points, persistent grids
// (layer 1: four CTAs per SM; layers 2 and 3: two, each with two A buffers).
static void conv_geometry(of_grid* g, int& nseg, int& lseg, long long& tiles) {
    nseg = (g->d.n1 + tc::M - 1) / tc::M;
    lseg = (g->d.n1 + nseg - 1) / nseg;
    tiles = (long long)g->d.n2 * g->d.n3 * nseg;
    OF_REQUIRE(tiles < (1LL << 31) - 4LL * num_sms(), OF_EINVAL,
               "grid too large for the network kernels (%lld row segments)", tiles);
}

// BWD: the data gradient (the kernel's weights P are then the backward array, its input the
// gradient of the layer above, zin the forward pre-activation and gout the FP32 output)
template <bool BWD = false>
static void launch_conv1_tc(of_grid* g, const float* r, const __nv_bfloat16* P, __nv_bfloat16* z1,
                            __nv_bfloat16* a1, float* rn, const double* rms, float sgn,
                            unsigned long long wait_ns, const __nv_bfloat16* zin = nullptr,
                            float* gout = nullptr) {
    static int configured_device = -1;
    if (configured_device != g->device) {
        OF_CUDA(cudaFuncSetAttribute(k_conv1_tc<BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM1));
        configured_device = g->device;
    }
    int nseg, lseg;
    long long tiles;
    conv_geometry(g, nseg, lseg, tiles);
    const int grid = (int)std::max(1LL, std::min(tiles, 4LL * num_sms()));
    launch_smem(k_conv1_tc<BWD>, grid, tc::THREADS, tc::SMEM1, g->stream, g->d, nseg, lseg, r, P, z1, a1,
                rn, rms, sgn, g->s.scalars + SC_NET_ERR, wait_ns, zin, gout);
}

template <int LAYER, bool BWD = false>
static void launch_conv_tc(of_grid* g, const __nv_bfloat16* in, const __nv_bfloat16* P,
                           __nv_bfloat16* zout, __nv_bfloat16* aout, float* y, const double* s_dev,
                           unsigned long long wait_ns, const __nv_bfloat16* zin = nullptr,
                           float* gout = nullptr) {
    static int configured_device = -1;
    if (configured_device != g->device) {
        OF_CUDA(cudaFuncSetAttribute(k_conv_tc<LAYER, BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tc::SMEM));
        configured_device = g->device;
    }
    int nseg, lseg;
    long long tiles;
    conv_geometry(g, nseg, lseg, tiles);
    const int grid = (int)std::max(1LL, std::min(tiles, 2LL * num_sms()));
    launch_smem(k_conv_tc<LAYER, BWD>, grid, tc::THREADS, tc::SMEM, g->stream, g->d, nseg, lseg, in, P,
                zout, aout, y, s_dev, g->s.scalars + SC_NET_ERR, wait_ns, zin, gout);
}

// algorithmic bytes of one application: r read by the RMS pass and by layer 1, a1 and a2
// (16 BF16 channels) written once and read once, z written
static double net_bytes(long long n) { return (double)n * (4.0 + 4.0 + 4 * 32.0 + 4.0); }

// out = s net(r / s) (apply) or net(r / s) with the activations kept (training)
static void net_forward(of_grid* g, of_precond* P, const float* r, float* out, const NetBufs& B,
                        bool training, float sgn = 1.f) {
    const long long n = g->d.n;
    ProfScope ps(g, PC_NET, net_bytes(n));
    const double* rms = g->s.scalars + SC_NET + 1;
    launch(k_rms32, vec_blocks(n), 256, g->stream, n, r, red_ctx(g, SC_NET));
    const __nv_bfloat16* W = P->pbf;
    launch_conv1_tc(g, r, W, training ? B.z1 : nullptr, B.a1, training ? B.rn : nullptr, rms, sgn,
                    P->wait_ns);
    launch_conv_tc<2>(g, B.a1, W, training ? B.z2 : nullptr, B.a2, nullptr, nullptr, P->wait_ns);
    launch_conv_tc<3>(g, B.a2, W, nullptr, nullptr, out, training ? nullptr : rms, P->wait_ns);
}

// loss sums (scalars 112, 113) and gradient accumulation (scaled) for one residual, taken
// with sign sgn
static void net_loss_grad(of_grid* g, of_precond* P, const float* r, const NetBufs& B, float gscale,
                          float sgn = 1.f) {
    const long long n = g->d.n;
    net_forward(g, P, r, B.y, B, true, sgn);
    launch_stencil<float, 2>(g, g->w32, OpNegLap32{B.y, B.Ay, (float)P->shift});
    launch(k_net_loss, vec_blocks(n), 256, g->stream, n, (const float*)B.y, (const float*)B.Ay,
           (const float*)B.rn, B.gy, red_ctx(g, SC_NET + 2));
    // data gradients on the tensor cores (BF16 operands, FP32 accumulation): gz2 from gy with
    // the mirrored W3, gz1 from gz2 with the transposed, mirrored W2
    launch(k_backward_weights, (NPAR + 255) / 256, 256, g->stream, (const __nv_bfloat16*)P->pbf, P->pbw);
    launch_conv1_tc<true>(g, B.gy, P->pbw, nullptr, B.gz2b, nullptr, nullptr, 1.f, P->wait_ns, B.z2, B.gz2);
    launch_conv_tc<2, true>(g, B.gz2b, P->pbw, nullptr, nullptr, nullptr, nullptr, P->wait_ns, B.z1, B.gz1);
    launch(k_net_wgrad, B.wblocks, 256, g->stream, g->d, (const float*)B.rn, (const __nv_bfloat16*)B.a1,
           (const __nv_bfloat16*)B.a2, (const float*)B.gz1, (const float*)B.gz2, (const float*)B.gy,
           B.part);
    launch(k_sum_parts, (NPAR + 255) / 256, 256, g->stream, B.wblocks, (const float*)B.part, P->grad,
           gscale);
}

static void require_device(of_grid* g, of_precond* P) {
    OF_REQUIRE(P->device == g->device, OF_EINVAL, "preconditioner made on device %d, grid on device %d",
               P->device, g->device);
}

struct Sink {
    float* buf;
    int stride, max_samples, count;
};

// Flexible CG on the FP32 inner system A x = r, A = -L_h + shift (x = 0 on entry; the KState
// at st_off holds rr, tol2, maxit, done).  P == nullptr: every step is plain (Jacobi) CG.
// Buffers r (overwritten), ra and z of n floats; the direction ring lives in the grid's
// workspace.  With a sink, every stride-th residual (the initial one first) is copied to
// sink->buf[k * n], up to max_samples.
KState iterate_fcg(of_grid* g, of_precond* P, double theta, int st_off, float* x, float* r,
                   float* ra, float* z, int check_every, Sink* sink, double* net_steps,
                   double shift) {
    const long long n = g->d.n;
    KState* st = kstate(g, st_off);
    FState* fs = fstate(g);
    const bool net = P != nullptr;
    NetBufs B{};
    if (net) {
        require_device(g, P);
        B = net_bufs(g, false);
    }
    const size_t vec = al256((size_t)n * sizeof(float));
    char* rb = (char*)ws(g, WS_K5, 2 * FCG_M * vec);
    Ring ring;
    for (int j = 0; j < FCG_M; ++j) {
        ring.p[j] = (float*)(rb + (2 * j) * vec);
        ring.Ap[j] = (float*)(rb + (2 * j + 1) * vec);
    }
    const int nb = vec_blocks(n);
    auto take_sample = [&](const float* v) {
        OF_CUDA(cudaMemcpyAsync(sink->buf + (long long)sink->count * n, v, sizeof(float) * n,
                                cudaMemcpyDeviceToDevice, g->stream));
        ++sink->count;
    };
    launch(k_fcg_reset, 1, 1, g->stream, fs);
    if (net) net_reset_error(g);
    if (sink && sink->count < sink->max_samples) take_sample(r);
    if (net) net_forward(g, P, r, z, B, false);
    const int project = shift == 0.0;
    launch(k_fcg_dots, nb, 256, g->stream, n, (const float*)r, (const float*)z, (int)net, project, theta,
           ring, 0, st, fs, red_ctx(g, FDOTS_OFF));
    launch(k_fcg_direction, nb, 256, g->stream, n, (const float*)r, (const float*)z, ring, 0, ring.p[0],
           (const KState*)st, (const FState*)fs);
    float* rc = r;
    float* rn = ra;
    const int every = std::max(1, check_every);
    KState h;
    for (int it = 1;; ++it) {
        const int slot = (it - 1) % FCG_M;
        launch_stencil<float, 2>(g, g->w32, OpFcgA{ring.p[slot], rc, ring.Ap[slot], st, fs, slot,
                                                   red_ctx(g, 0), (float)shift});
        {
            ProfScope ps(g, PC_UPDATE, 5.0 * 4.0 * (double)n);
            launch(k_fcg_update, nb, 256, g->stream, n, x, (const float*)rc, rn, (const float*)ring.p[slot],
                   (const float*)ring.Ap[slot], st, red_ctx(g, 0));
        }
        if (sink && sink->count < sink->max_samples && it % sink->stride == 0) {
            fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);   // only while still iterating
            if (h.iters == (double)it) take_sample(rn);
        }
        const int valid = std::min(it, FCG_M);
        if (net) net_forward(g, P, rn, z, B, false);
        launch(k_fcg_dots, nb, 256, g->stream, n, (const float*)rn, (const float*)z, (int)net, project,
               theta, ring, valid, st, fs, red_ctx(g, FDOTS_OFF));
        launch(k_fcg_direction, nb, 256, g->stream, n, (const float*)rn, (const float*)z, ring, valid,
               ring.p[it % FCG_M], (const KState*)st, (const FState*)fs);
        std::swap(rc, rn);
        if (it % every == 0) {
            fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
            if (h.done != 0.0) break;
        }
    }
    if (net) net_check_error(g);
    if (net_steps) {
        FState f;
        fetch_scalars(g, FS_OFF, sizeof(FState) / sizeof(double), (double*)&f);
        *net_steps += f.net_steps;
    }
    return h;
}

KState iterate_fgmres(of_grid* g, of_precond* P, double theta, int st_off, float2* x, const float2* b,
                      float* z, float* rs, float a, double2 Q, double* net_steps) {
    using cplx = std::complex<double>;
    const long long n = g->d.n;
    KState h;
    fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);   // |b|^2, tol2, maxit (x = 0)
    h.iters = 0.0;
    h.breakdown = 0.0;
    if (!(h.rr > h.tol2)) {
        h.done = 1.0;
        return h;
    }
    if (P) require_device(g, P);
    const size_t vec = al256((size_t)n * sizeof(float2));
    char* base = (char*)ws(g, WS_FGM, (2 * GM_M + 3) * vec);
    VecSet V, Zs;
    for (int k = 0; k <= GM_M; ++k) V.v[k] = (float2*)(base + k * vec);
    for (int k = 0; k < GM_M; ++k) Zs.v[k] = (float2*)(base + (GM_M + 1 + k) * vec);
    Zs.v[GM_M] = nullptr;
    float2* W = (float2*)(base + (2 * GM_M + 1) * vec);
    float* scr = (float*)(base + (2 * GM_M + 2) * vec);   // two fields of n floats
    const int nb = vec_blocks(n);
    const int maxit = (int)h.maxit;
    double* sc = g->s.scalars;
    const double c = std::sqrt((double)Q.x * Q.x + (double)Q.y * Q.y) / a;   // A_r = -L_h + c
    double beta = std::sqrt(h.rr), rr = h.rr;
    launch(k_gm_scale, nb, 256, g->stream, n, b, V.v[0], (float)(1.0 / beta));
    int it = 0, inner = 0;
    for (;;) {   // one restart cycle
        cplx H[GM_M + 1][GM_M] = {};
        cplx cs[GM_M], sn[GM_M], gv[GM_M + 1] = {};
        gv[0] = beta;
        VecSet Zc{};
        int k = 0;
        for (int j = 0; j < GM_M; ++j) {
            // z_j: flexible CG with the network on A_r z = v_j, real and imaginary parts
            launch(k_split2, nb, 256, g->stream, n, (const float2*)V.v[j], rs);
            for (int part = 0; part < 2; ++part) {
                float* rp = rs + part * n;
                float* zp = z + part * n;
                launch(k_nest_init, nb, 256, g->stream, n, (const float*)rp, zp, GM_TAU, GM_INNER_MAX,
                       kstate(g, KS_NEST), red_ctx(g, 0));
                const KState hn = iterate_fcg(g, P, theta, KS_NEST, zp, rp, scr, scr + n, 4, nullptr,
                                              net_steps, c);
                inner += (int)hn.iters;
            }
            launch(k_merge2, nb, 256, g->stream, n, (const float*)z, Zs.v[j]);
            float2* zj = Zs.v[j];
            Zc.v[j] = zj;
            launch_stencil<float2, 1>(g, g->w32, OpGmA{zj, W, a, Q});
            {
                ProfScope ps(g, PC_UPDATE, 4.0 * 8.0 * (j + 2) * (double)n);
                launch(k_gm_dots, nb, 256, g->stream, n, (const float2*)W, V, j + 1, red_ctx(g, GH1));
                launch(k_gm_orth, nb, 256, g->stream, n, W, V, j + 1, (const double*)(sc + GH1), 0, red_ctx(g, GNRM));
                launch(k_gm_dots, nb, 256, g->stream, n, (const float2*)W, V, j + 1, red_ctx(g, GH2));
                launch(k_gm_orth, nb, 256, g->stream, n, W, V, j + 1, (const double*)(sc + GH2), 1, red_ctx(g, GNRM));
            }
            double hv[4 * GM_M + 1];
            fetch_scalars(g, GH1, 4 * GM_M + 1, hv);
            for (int i = 0; i <= j; ++i)
                H[i][j] = cplx(hv[2 * i] + hv[2 * GM_M + 2 * i], hv[2 * i + 1] + hv[2 * GM_M + 2 * i + 1]);
            const double hn = std::sqrt(std::max(hv[4 * GM_M], 0.0));
            H[j + 1][j] = hn;
            // the earlier rotations on the new column, then one that zeroes H[j+1][j]
            for (int i = 0; i < j; ++i) {
                const cplx t = cs[i] * H[i][j] + sn[i] * H[i + 1][j];
                H[i + 1][j] = -std::conj(sn[i]) * H[i][j] + cs[i] * H[i + 1][j];
                H[i][j] = t;
            }
            const double aa = std::abs(H[j][j]);
            if (hn == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else if (aa == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                const double t = std::hypot(aa, hn);
                cs[j] = aa / t;
                sn[j] = (H[j][j] / aa) * hn / t;
            }
            H[j][j] = cs[j] * H[j][j] + sn[j] * H[j + 1][j];
            H[j + 1][j] = 0.0;
            gv[j + 1] = -std::conj(sn[j]) * gv[j];
            gv[j] = cs[j] * gv[j];
            ++it;
            k = j + 1;
            const double est2 = std::norm(gv[j + 1]);
            if (!std::isfinite(est2) || !std::isfinite(hn)) {
                h.breakdown = 1.0;
                break;
            }
            if (est2 <= h.tol2 || hn == 0.0 || it >= maxit) break;
            launch(k_gm_scale, nb, 256, g->stream, n, (const float2*)W, V.v[j + 1], (float)(1.0 / hn));
        }
        // x += Z y, y from the triangular system R y = g
        GmCoef y{};
        cplx yc[GM_M];
        for (int i = k - 1; i >= 0; --i) {
            cplx s = gv[i];
            for (int l = i + 1; l < k; ++l) s -= H[i][l] * yc[l];
            if (std::abs(H[i][i]) == 0.0) {
                h.breakdown = 1.0;
                yc[i] = 0.0;
            } else {
                yc[i] = s / H[i][i];
            }
            if (!std::isfinite(std::abs(yc[i]))) {
                h.breakdown = 1.0;
                yc[i] = 0.0;
            }
        }
        for (int i = 0; i < k; ++i) y.y[i] = make_double2(yc[i].real(), yc[i].imag());
        launch(k_gm_xupdate, nb, 256, g->stream, n, x, Zc, k, y);
        // the true residual of the inner system restarts the next cycle
        launch_stencil<float2, 1>(g, g->w32, OpGmResid{(const float2*)x, b, W, a, Q, red_ctx(g, GNRM), 0.f});
        fetch_scalars(g, GNRM, 1, &rr);
        if (!(rr > h.tol2) || it >= maxit || h.breakdown != 0.0 || !std::isfinite(rr)) break;
        beta = std::sqrt(rr);
        launch(k_gm_scale, nb, 256, g->stream, n, (const float2*)W, V.v[0], (float)(1.0 / beta));
    }
    h.iters = it + inner;
    h.rr = rr;
    h.done = 1.0;
    return h;
}

}  // namespace of

using namespace of;

extern "C" {

int of_precond_num_params(void) { return NPAR; }

of_status of_precond_create(const float* params, int nparams, of_precond** out) {
    if (!params || nparams != NPAR || !out) {
        set_error("of_precond_create: need %d parameters and an output pointer", NPAR);
        return OF_EINVAL;
    }
    of_precond* P = new (std::nothrow) of_precond();
    if (!P) return OF_ENOMEM;
    try {
        OF_CUDA(cudaGetDevice(&P->device));
        OF_CUDA(cudaMalloc(&P->params, sizeof(float) * NPAR * 4));
        OF_CUDA(cudaMalloc(&P->pbf, sizeof(__nv_bfloat16) * NPAR));
        OF_CUDA(cudaMalloc(&P->pbw, sizeof(__nv_bfloat16) * NPAR));
        note_resource();
        note_resource();
        note_resource();
        P->grad = P->params + NPAR;
        P->m = P->params + 2 * NPAR;
        P->v = P->params + 3 * NPAR;
        OF_CUDA(cudaMemcpy(P->params, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
        OF_CUDA(cudaMemset(P->grad, 0, sizeof(float) * NPAR * 3));
        launch(k_to_bf16, (NPAR + 255) / 256, 256, (cudaStream_t)0, NPAR, (const float*)P->params, P->pbf);
        OF_CUDA(cudaDeviceSynchronize());
        *out = P;
        return OF_OK;
    } catch (...) {
        if (P->params) cudaFree(P->params);
        if (P->pbf) cudaFree(P->pbf);
        if (P->pbw) cudaFree(P->pbw);
        delete P;
        try {
            throw;
        } catch (const Error& e) {
            return e.code;
        } catch (...) {
            return unexpected_exception();
        }
    }
}

of_status of_precond_set_shift(of_precond* P, double shift) {
    if (!P || !(shift >= 0.0) || !std::isfinite(shift)) {
        set_error("of_precond_set_shift: need a handle and a finite shift >= 0");
        return OF_EINVAL;
    }
    P->shift = shift;
    return OF_OK;
}

of_status of_precond_destroy(of_precond* P) {
    if (!P) return OF_OK;
    cudaDeviceSynchronize();
    cudaFree(P->params);
    cudaFree(P->pbf);
    cudaFree(P->pbw);
    delete P;
    return OF_OK;
}

of_status of_precond_set_wait_limit(of_precond* P, double seconds) {
    if (!P || !(seconds >= 0.0) || seconds > 60.0) {
        set_error("of_precond_set_wait_limit: need a handle and 0 <= seconds <= 60");
        return OF_EINVAL;
    }
    P->wait_ns = (unsigned long long)(seconds * 1e9);
    return OF_OK;
}

of_status of_precond_get_params(of_precond* P, float* params, int nparams) {
    if (!P || !params || nparams != NPAR) {
        set_error("of_precond_get_params: need %d parameters", NPAR);
        return OF_EINVAL;
    }
    try {
        OF_CUDA(cudaDeviceSynchronize());
        OF_CUDA(cudaMemcpy(params, P->params, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_precond_apply(of_grid* g, of_precond* P, const float* r, float* z) {
    if (!g || !P || !r || !z || r == z) {
        set_error("of_precond_apply: null argument or r == z");
        return OF_EINVAL;
    }
    try {
        require_device(g, P);
        NetBufs B = net_bufs(g, false);
        net_reset_error(g);
        net_forward(g, P, r, z, B, false);
        net_check_error(g);
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_precond_loss_grad(of_grid* g, of_precond* P, const float* r, double* loss, float* grad) {
    if (!g || !P || !r) {
        set_error("of_precond_loss_grad: null argument");
        return OF_EINVAL;
    }
    try {
        require_device(g, P);
        NetBufs B = net_bufs(g, true);
        OF_CUDA(cudaMemsetAsync(P->grad, 0, sizeof(float) * NPAR, g->stream));
        net_reset_error(g);
        net_loss_grad(g, P, r, B, 1.f);
        net_check_error(g);
        double s[2];
        fetch_scalars(g, SC_NET + 2, 2, s);
        if (loss) *loss = 0.5 * s[0] - s[1];
        if (grad) OF_CUDA(cudaMemcpy(grad, P->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
        OF_CUDA(cudaMemsetAsync(P->grad, 0, sizeof(float) * NPAR, g->stream));
        OF_CUDA(cudaStreamSynchronize(g->stream));
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_precond_train(of_grid* g, of_precond* P, const float* samples, int nsamples,
                           const int* order, int steps, int batch, float lr, double* loss_out) {
    if (!g || !P || !samples || !order || nsamples < 1 || steps < 1 || batch < 1 || !(lr > 0.f)) {
        set_error("of_precond_train: bad argument");
        return OF_EINVAL;
    }
    for (long long k = 0; k < (long long)steps * batch; ++k)
        if (order[k] < 0 || order[k] >= nsamples) {
            set_error("of_precond_train: order[%lld] = %d outside [0, %d)", k, order[k], nsamples);
            return OF_EINVAL;
        }
    try {
        require_device(g, P);
        NetBufs B = net_bufs(g, true);
        const long long n = g->d.n;
        double last = 0.0;
        net_reset_error(g);
        for (int s = 0; s < steps; ++s) {
            const bool final_step = s == steps - 1;
            double lsum = 0.0;
            for (int k = 0; k < batch; ++k) {
                // residuals have no preferred sign: every other visit trains on -r
                const float sgn = ((s * batch + k) & 1) ? -1.f : 1.f;
                net_loss_grad(g, P, samples + (long long)order[s * batch + k] * n, B, 1.f / batch, sgn);
                if (final_step) {
                    double v[2];
                    fetch_scalars(g, SC_NET + 2, 2, v);
                    lsum += 0.5 * v[0] - v[1];
                }
            }
            P->step += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)P->step);
            const float c2 = 1.f - std::pow(b2, (float)P->step);
            launch(k_adam, (NPAR + 255) / 256, 256, g->stream, P->params, P->pbf, P->grad, P->m, P->v, lr,
                   b1, b2, c1, c2);
            if (final_step) last = lsum / batch;
        }
        net_check_error(g);
        if (loss_out) *loss_out = last / (double)n;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_precond_collect(of_grid* g, const double* rho, double shift, int stride,
                             int max_samples, float* samples, int* count) {
    if (!g || !rho || stride < 1 || max_samples < 1 || !samples || !count || !(shift >= 0.0) ||
        !std::isfinite(shift)) {
        set_error("of_precond_collect: bad argument");
        return OF_EINVAL;
    }
    try {
        const long long n = g->d.n;
        Arena ar = arena(g);
        if (shift == 0.0) {
            launch(k_sum_product, vec_blocks(n), 256, g->stream, n, rho, (const double*)nullptr,
                   red_ctx(g, 120));
            launch(k_form_rhs, vec_blocks(n), 256, g->stream, n, rho, (const double*)nullptr,
                   (const double*)(g->s.scalars + 120), 4.0 * M_PI, (double*)ar.b64);
        } else {
            OF_CUDA(cudaMemcpyAsync(ar.b64, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
        }
        launch(k_sumsq64, vec_blocks(n), 256, g->stream, n, (const double*)ar.b64, red_ctx(g, 121));
        const long long maxit = std::min<long long>(20000, (long long)stride * max_samples);
        launch(k_unit32, vec_blocks(n), 256, g->stream, n, (const double*)ar.b64, (float*)ar.r32,
               (float*)ar.e32, (const double*)(g->s.scalars + 121), 1e-6, (int)maxit, kstate(g, KS32),
               red_ctx(g, 0));
        Sink sink{samples, stride, max_samples, 0};
        iterate_fcg(g, nullptr, 0.0, KS32, (float*)ar.e32, (float*)ar.r32, (float*)ar.pa32,
                    (float*)ar.z32, 8, &sink, nullptr, shift);
        OF_CUDA(cudaStreamSynchronize(g->stream));
        *count = sink.count;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

}  // extern "C"
