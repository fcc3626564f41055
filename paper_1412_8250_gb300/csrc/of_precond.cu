// Learned preconditioner for the Poisson CG.
//
// Network: three periodic 3x3x3 convolutions, 1 -> 16 -> 16 -> 1 channels with biases, exact
// (erf) GELU after the first two; weights and stored activations in BF16, every sum in FP32.
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

__device__ __forceinline__ void load16(const __nv_bfloat16* p, float (&v)[NC]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 u0 = __ldg(q), u1 = __ldg(q + 1);
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

__device__ __forceinline__ void store16(__nv_bfloat16* p, const float (&v)[NC]) {
    uint4 u0, u1;
    __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&u0);
    __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&u1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h0[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        h1[k] = __floats2bfloat162_rn(v[8 + 2 * k], v[8 + 2 * k + 1]);
    }
    uint4* q = reinterpret_cast<uint4*>(p);
    q[0] = u0;
    q[1] = u1;
}

// ---------------------------------------------------------------- forward
// layer 1: z1 = W1 * (sgn r / s) + b1, a1 = GELU(z1); also rn = sgn r / s (training only)
__global__ void __launch_bounds__(256) k_net_l1(Dims d, const float* __restrict__ r, const double* rms_dev,
                                                float sgn, const __nv_bfloat16* __restrict__ P,
                                                __nv_bfloat16* z1, __nv_bfloat16* a1, float* rn) {
    __shared__ float W[NT * NC + NC];   // [t][o], then b1
    for (int k = threadIdx.x; k < NT * NC; k += blockDim.x)
        W[k] = __bfloat162float(P[OW1 + (k % NC) * NT + k / NC]);
    for (int k = threadIdx.x; k < NC; k += blockDim.x) W[NT * NC + k] = __bfloat162float(P[OB1 + k]);
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const double rms = *rms_dev;
    const float inv = rms > 0.0 ? sgn * (float)(1.0 / rms) : 0.f;
    const Nb nb = neighbours(d, i);
    float acc[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) acc[o] = W[NT * NC + o];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float v = __ldg(r + nb.at(t)) * inv;
#pragma unroll
        for (int o = 0; o < NC; ++o) acc[o] = fmaf(W[t * NC + o], v, acc[o]);
    }
    if (rn) rn[i] = r[i] * inv;
    float g[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) g[o] = gelu_f(acc[o]);
    if (z1) store16(z1 + i * NC, acc);
    store16(a1 + i * NC, g);
}

// layer 2: z2 = W2 * a1 + b2, a2 = GELU(z2); W2 staged as [t][c][o]
__global__ void __launch_bounds__(256) k_net_l2(Dims d, const __nv_bfloat16* __restrict__ a1,
                                                const __nv_bfloat16* __restrict__ P,
                                                __nv_bfloat16* z2, __nv_bfloat16* a2) {
    __shared__ __align__(16) float W[NT * NC * NC + NC];
    for (int k = threadIdx.x; k < NT * NC * NC; k += blockDim.x) {
        const int t = k / (NC * NC), c = (k / NC) % NC, o = k % NC;
        W[k] = __bfloat162float(P[OW2 + (o * NC + c) * NT + t]);
    }
    for (int k = threadIdx.x; k < NC; k += blockDim.x) W[NT * NC * NC + k] = __bfloat162float(P[OB2 + k]);
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const Nb nb = neighbours(d, i);
    float acc[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) acc[o] = W[NT * NC * NC + o];
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
        float v[NC];
        load16(a1 + nb.at(t) * NC, v);
        const float4* Wt = reinterpret_cast<const float4*>(W + t * NC * NC);
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int q = 0; q < NC / 4; ++q) {
                const float4 w = Wt[c * (NC / 4) + q];
                acc[4 * q] = fmaf(w.x, v[c], acc[4 * q]);
                acc[4 * q + 1] = fmaf(w.y, v[c], acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(w.z, v[c], acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(w.w, v[c], acc[4 * q + 3]);
            }
    }
    float g[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) g[o] = gelu_f(acc[o]);
    if (z2) store16(z2 + i * NC, acc);
    store16(a2 + i * NC, g);
}

// layer 3: y = scale (W3 * a2 + b3), scale = s (application) or 1 (training)
__global__ void __launch_bounds__(256) k_net_l3(Dims d, const __nv_bfloat16* __restrict__ a2,
                                                const __nv_bfloat16* __restrict__ P, const double* s_dev,
                                                float* y) {
    __shared__ __align__(16) float W[NT * NC + 1];   // [t][c], then b3
    for (int k = threadIdx.x; k < NT * NC; k += blockDim.x)
        W[k] = __bfloat162float(P[OW3 + (k % NC) * NT + k / NC]);
    if (threadIdx.x == 0) W[NT * NC] = __bfloat162float(P[OB3]);
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const Nb nb = neighbours(d, i);
    float acc = W[NT * NC];
#pragma unroll 3
    for (int t = 0; t < NT; ++t) {
        float v[NC];
        load16(a2 + nb.at(t) * NC, v);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc = fmaf(W[t * NC + c], v[c], acc);
    }
    const float scale = s_dev ? (float)*s_dev : 1.f;
    y[i] = scale * acc;
}

// ---------------------------------------------------------------- backward
// gz2[x][c] = GELU'(z2[x][c]) sum_t W3[c][t] gy[x - t]
__global__ void __launch_bounds__(256) k_net_l3_bwd(Dims d, const float* __restrict__ gy,
                                                    const __nv_bfloat16* __restrict__ z2,
                                                    const __nv_bfloat16* __restrict__ P, float* gz2) {
    __shared__ float W[NT * NC];   // [t][c]
    for (int k = threadIdx.x; k < NT * NC; k += blockDim.x)
        W[k] = __bfloat162float(P[OW3 + (k % NC) * NT + k / NC]);
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const Nb nb = neighbours(d, i);
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float g = __ldg(gy + nb.at(NT - 1 - t));   // x - t is the mirrored tap
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(W[t * NC + c], g, acc[c]);
    }
    float z[NC];
    load16(z2 + i * NC, z);
    float4* out = reinterpret_cast<float4*>(gz2 + i * NC);
#pragma unroll
    for (int q = 0; q < NC / 4; ++q)
        out[q] = make_float4(acc[4 * q] * gelu_grad_f(z[4 * q]), acc[4 * q + 1] * gelu_grad_f(z[4 * q + 1]),
                             acc[4 * q + 2] * gelu_grad_f(z[4 * q + 2]),
                             acc[4 * q + 3] * gelu_grad_f(z[4 * q + 3]));
}

// gz1[x][c] = GELU'(z1[x][c]) sum_t sum_o W2[o][c][t] gz2[x - t][o]; W2 staged as [t][o][c]
__global__ void __launch_bounds__(256) k_net_l2_bwd(Dims d, const float* __restrict__ gz2,
                                                    const __nv_bfloat16* __restrict__ z1,
                                                    const __nv_bfloat16* __restrict__ P, float* gz1) {
    __shared__ __align__(16) float W[NT * NC * NC];
    for (int k = threadIdx.x; k < NT * NC * NC; k += blockDim.x) {
        const int t = k / (NC * NC), o = (k / NC) % NC, c = k % NC;
        W[k] = __bfloat162float(P[OW2 + (o * NC + c) * NT + t]);
    }
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const Nb nb = neighbours(d, i);
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
        const float4* g4 = reinterpret_cast<const float4*>(gz2 + nb.at(NT - 1 - t) * NC);
        const float4* Wt = reinterpret_cast<const float4*>(W + t * NC * NC);
#pragma unroll
        for (int oq = 0; oq < NC / 4; ++oq) {
            const float4 gq = __ldg(g4 + oq);
            const float go[4] = {gq.x, gq.y, gq.z, gq.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = 4 * oq + k;
#pragma unroll
                for (int q = 0; q < NC / 4; ++q) {
                    const float4 w = Wt[o * (NC / 4) + q];
                    acc[4 * q] = fmaf(w.x, go[k], acc[4 * q]);
                    acc[4 * q + 1] = fmaf(w.y, go[k], acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(w.z, go[k], acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(w.w, go[k], acc[4 * q + 3]);
                }
            }
        }
    }
    float z[NC];
    load16(z1 + i * NC, z);
    float4* out = reinterpret_cast<float4*>(gz1 + i * NC);
#pragma unroll
    for (int q = 0; q < NC / 4; ++q)
        out[q] = make_float4(acc[4 * q] * gelu_grad_f(z[4 * q]), acc[4 * q + 1] * gelu_grad_f(z[4 * q + 1]),
                             acc[4 * q + 2] * gelu_grad_f(z[4 * q + 2]),
                             acc[4 * q + 3] * gelu_grad_f(z[4 * q + 3]));
}

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
                s_a1[p][c] = j >= 0 ? __bfloat162float(a1[j * NC + c]) : 0.f;
                s_a2[p][c] = j >= 0 ? __bfloat162float(a2[j * NC + c]) : 0.f;
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
    float acc[2];
    __device__ bool begin() {
        if (st->done != 0.0) return false;
        acc[0] = acc[1] = 0.f;
        return true;
    }
    __device__ float load(long long i) const { return p[i]; }
    __device__ void store(long long i, float c, float lap) {
        Ap[i] = -lap;
        acc[0] = fmaf(c, -lap, acc[0]);
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
// when cos(r, d) > theta, else d = r, and sets c_j = d.Ap_j / p_j.Ap_j (sum Ap_j = 0 for the
// Laplacian, so the mean shift drops out of d.Ap_j).
constexpr int DOTS_K = 4 + 2 * FCG_M;
__global__ void __launch_bounds__(256) k_fcg_dots(long long n, const float* __restrict__ r,
                                                  const float* __restrict__ z, int has_net, double theta,
                                                  Ring ring, int valid, KState* st, FState* fs, RedCtx rc) {
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
            mean = acc[0] / (double)n;
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
    __nv_bfloat16 *a1, *a2, *z1, *z2;
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
    const size_t bytes = training ? 4 * act + 4 * f1 + 2 * f16 + al256((size_t)wb * NPAR * 4) : 2 * act;
    char* p = (char*)ws(g, WS_K6, bytes);
    NetBufs B{};
    B.a1 = (__nv_bfloat16*)p; p += act;
    B.a2 = (__nv_bfloat16*)p; p += act;
    B.wblocks = wb;
    if (!training) return B;
    B.z1 = (__nv_bfloat16*)p; p += act;
    B.z2 = (__nv_bfloat16*)p; p += act;
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
struct OpNegLap32 {
    const float* x;
    float* y;
    __device__ bool begin() { return true; }
    __device__ float load(long long i) const { return x[i]; }
    __device__ void store(long long i, float, float lap) { y[i] = -lap; }
    __device__ void end() {}
};

static inline unsigned pt_blocks(long long n) { return (unsigned)((n + 255) / 256); }

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
    launch(k_net_l1, pt_blocks(n), 256, g->stream, g->d, r, rms, sgn, (const __nv_bfloat16*)P->pbf,
           training ? B.z1 : nullptr, B.a1, training ? B.rn : nullptr);
    launch(k_net_l2, pt_blocks(n), 256, g->stream, g->d, (const __nv_bfloat16*)B.a1,
           (const __nv_bfloat16*)P->pbf, training ? B.z2 : nullptr, B.a2);
    launch(k_net_l3, pt_blocks(n), 256, g->stream, g->d, (const __nv_bfloat16*)B.a2,
           (const __nv_bfloat16*)P->pbf, training ? nullptr : rms, out);
}

// loss sums (scalars 112, 113) and gradient accumulation (scaled) for one residual, taken
// with sign sgn
static void net_loss_grad(of_grid* g, of_precond* P, const float* r, const NetBufs& B, float gscale,
                          float sgn = 1.f) {
    const long long n = g->d.n;
    net_forward(g, P, r, B.y, B, true, sgn);
    launch_stencil<float, 2>(g, g->w32, OpNegLap32{B.y, B.Ay});
    launch(k_net_loss, vec_blocks(n), 256, g->stream, n, (const float*)B.y, (const float*)B.Ay,
           (const float*)B.rn, B.gy, red_ctx(g, SC_NET + 2));
    launch(k_net_l3_bwd, pt_blocks(n), 256, g->stream, g->d, (const float*)B.gy,
           (const __nv_bfloat16*)B.z2, (const __nv_bfloat16*)P->pbf, B.gz2);
    launch(k_net_l2_bwd, pt_blocks(n), 256, g->stream, g->d, (const float*)B.gz2,
           (const __nv_bfloat16*)B.z1, (const __nv_bfloat16*)P->pbf, B.gz1);
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

// Flexible CG on the FP32 inner system A x = r (x = 0 on entry; the KState at st_off holds
// rr, tol2, maxit, done).  P == nullptr: every step is plain (Jacobi) CG.  Buffers r
// (overwritten), ra and z of n floats; the direction ring lives in the grid's workspace.  With
// a sink, every stride-th residual (the initial one first) is copied to sink->buf[k * n], up
// to max_samples.
KState iterate_fcg(of_grid* g, of_precond* P, double theta, int st_off, float* x, float* r,
                   float* ra, float* z, int check_every, Sink* sink, double* net_steps) {
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
    if (sink && sink->count < sink->max_samples) take_sample(r);
    if (net) net_forward(g, P, r, z, B, false);
    launch(k_fcg_dots, nb, 256, g->stream, n, (const float*)r, (const float*)z, (int)net, theta, ring, 0,
           st, fs, red_ctx(g, 0));
    launch(k_fcg_direction, nb, 256, g->stream, n, (const float*)r, (const float*)z, ring, 0, ring.p[0],
           (const KState*)st, (const FState*)fs);
    float* rc = r;
    float* rn = ra;
    const int every = std::max(1, check_every);
    KState h;
    for (int it = 1;; ++it) {
        const int slot = (it - 1) % FCG_M;
        launch_stencil<float, 2>(g, g->w32, OpFcgA{ring.p[slot], rc, ring.Ap[slot], st, fs, slot,
                                                   red_ctx(g, 0)});
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
        launch(k_fcg_dots, nb, 256, g->stream, n, (const float*)rn, (const float*)z, (int)net, theta, ring,
               valid, st, fs, red_ctx(g, 0));
        launch(k_fcg_direction, nb, 256, g->stream, n, (const float*)rn, (const float*)z, ring, valid,
               ring.p[it % FCG_M], (const KState*)st, (const FState*)fs);
        std::swap(rc, rn);
        if (it % every == 0) {
            fetch_scalars(g, st_off, KSTATE_DOUBLES, (double*)&h);
            if (h.done != 0.0) break;
        }
    }
    if (net_steps) {
        FState f;
        fetch_scalars(g, FS_OFF, sizeof(FState) / sizeof(double), (double*)&f);
        *net_steps += f.net_steps;
    }
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
        P->grad = P->params + NPAR;
        P->m = P->params + 2 * NPAR;
        P->v = P->params + 3 * NPAR;
        OF_CUDA(cudaMemcpy(P->params, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
        OF_CUDA(cudaMemset(P->grad, 0, sizeof(float) * NPAR * 3));
        launch(k_to_bf16, (NPAR + 255) / 256, 256, (cudaStream_t)0, NPAR, (const float*)P->params, P->pbf);
        OF_CUDA(cudaDeviceSynchronize());
        *out = P;
        return OF_OK;
    } catch (const Error& e) {
        if (P->params) cudaFree(P->params);
        if (P->pbf) cudaFree(P->pbf);
        delete P;
        return e.code;
    }
}

of_status of_precond_destroy(of_precond* P) {
    if (!P) return OF_OK;
    cudaDeviceSynchronize();
    cudaFree(P->params);
    cudaFree(P->pbf);
    delete P;
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
        net_forward(g, P, r, z, B, false);
        OF_CUDA(cudaStreamSynchronize(g->stream));
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
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
        net_loss_grad(g, P, r, B, 1.f);
        double s[2];
        fetch_scalars(g, SC_NET + 2, 2, s);
        if (loss) *loss = 0.5 * s[0] - s[1];
        if (grad) OF_CUDA(cudaMemcpy(grad, P->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
        OF_CUDA(cudaMemsetAsync(P->grad, 0, sizeof(float) * NPAR, g->stream));
        OF_CUDA(cudaStreamSynchronize(g->stream));
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
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
        OF_CUDA(cudaStreamSynchronize(g->stream));
        if (loss_out) *loss_out = last / (double)n;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

of_status of_precond_collect(of_grid* g, const double* rho, int stride, int max_samples,
                             float* samples, int* count) {
    if (!g || !rho || stride < 1 || max_samples < 1 || !samples || !count) {
        set_error("of_precond_collect: bad argument");
        return OF_EINVAL;
    }
    try {
        const long long n = g->d.n;
        Arena ar = arena(g);
        launch(k_sum_product, vec_blocks(n), 256, g->stream, n, rho, (const double*)nullptr,
               red_ctx(g, 120));
        launch(k_form_rhs, vec_blocks(n), 256, g->stream, n, rho, (const double*)nullptr,
               (const double*)(g->s.scalars + 120), 4.0 * M_PI, (double*)ar.b64);
        launch(k_sumsq64, vec_blocks(n), 256, g->stream, n, (const double*)ar.b64, red_ctx(g, 121));
        const long long maxit = std::min<long long>(20000, (long long)stride * max_samples);
        launch(k_unit32, vec_blocks(n), 256, g->stream, n, (const double*)ar.b64, (float*)ar.r32,
               (float*)ar.e32, (const double*)(g->s.scalars + 121), 1e-6, (int)maxit, kstate(g, KS32),
               red_ctx(g, 0));
        Sink sink{samples, stride, max_samples, 0};
        iterate_fcg(g, nullptr, 0.0, KS32, (float*)ar.e32, (float*)ar.r32, (float*)ar.pa32,
                    (float*)ar.z32, 8, &sink, nullptr);
        OF_CUDA(cudaStreamSynchronize(g->stream));
        *count = sink.count;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

}  // extern "C"
