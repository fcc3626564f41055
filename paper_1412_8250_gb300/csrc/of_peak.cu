// Arithmetic peaks of this GPU's CUDA cores, measured: the denominators of the roofline for
// kernels bound by FP64 or FP32 arithmetic rather than by memory (the FP64 Laplacian sweeps of
// the refinement residuals).  Not an operation of the method.
#include "of_internal.cuh"

namespace of {
namespace {

constexpr int PEAK_CHAINS = 8;      // independent FMA chains per thread (hides the FMA latency)
constexpr int PEAK_UNROLL = 16;
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

__device__ double g_peak_sink;

// a <- a * b + c on PEAK_CHAINS independent chains, iters x PEAK_UNROLL times.  b and c come
// from the host so that nothing folds; the sum of the chains (positive) is stored only if it
// equals a negative value passed in, which keeps the chains alive without a store per thread.
template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T b, T c, int iters, T never) {
    T a[PEAK_CHAINS];
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = (T)(threadIdx.x + i) * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u) {
#pragma unroll
            for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) s += a[i];
    if (s == never) g_peak_sink = s;
}

// The same with packed FP32x2 FMAs (two lanes per instruction).
__global__ void __launch_bounds__(PEAK_THREADS) k_fma2_peak(float b, float c, int iters, float never) {
    unsigned long long a[PEAK_CHAINS], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) {
        const float lo = (float)(threadIdx.x + i) * c, hi = (float)(threadIdx.x + 2 * i) * c;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u) {
#pragma unroll
            for (int i = 0; i < PEAK_CHAINS; ++i)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(bb), "l"(cc));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
        s += lo + hi;
    }
    if (s == never) g_peak_sink = s;
}

}  // namespace
}  // namespace of

using namespace of;

extern "C" {

of_status of_alu_peak(int kind, void* stream, double* flop_per_s) {
    if (!flop_per_s) { set_error("of_alu_peak: flop_per_s is NULL"); return OF_EINVAL; }
    if (kind != OF_PEAK_F64 && kind != OF_PEAK_F32 && kind != OF_PEAK_F32X2) {
        set_error("of_alu_peak: kind %d not in {OF_PEAK_F64, OF_PEAK_F32, OF_PEAK_F32X2}", kind);
        return OF_EINVAL;
    }
    *flop_per_s = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    try {
        int dev = 0, sms = 0;
        OF_CUDA(cudaGetDevice(&dev));
        OF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int blocks = sms * PEAK_BLOCKS_PER_SM;
        // a few ms per launch at the nominal rates (FP64 ~1.2, FP32 ~80 TFLOP/s)
        const int iters = kind == OF_PEAK_F64 ? 64 : 4096;
        for (int k = 0; k < 2; ++k) {
            OF_CUDA(cudaEventCreate(&ev[k]));
            note_resource();
        }
        auto run = [&]() {
            if (kind == OF_PEAK_F64)
                launch(k_fma_peak<double>, blocks, PEAK_THREADS, s, 0.999999999, 1e-9, iters, -1.0);
            else if (kind == OF_PEAK_F32)
                launch(k_fma_peak<float>, blocks, PEAK_THREADS, s, 0.9999f, 1e-6f, iters, -1.0f);
            else
                launch(k_fma2_peak, blocks, PEAK_THREADS, s, 0.9999f, 1e-6f, iters, -1.0f);
        };
        run();   // warm-up
        float best = 0.f;
        for (int rep = 0; rep < 5; ++rep) {
            OF_CUDA(cudaEventRecord(ev[0], s));
            run();
            OF_CUDA(cudaEventRecord(ev[1], s));
            OF_CUDA(cudaEventSynchronize(ev[1]));
            float ms = 0.f;
            OF_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            if (rep == 0 || ms < best) best = ms;
        }
        const double lanes = kind == OF_PEAK_F32X2 ? 2.0 : 1.0;
        const double fmas = (double)blocks * PEAK_THREADS * PEAK_CHAINS * PEAK_UNROLL * iters * lanes;
        *flop_per_s = 2.0 * fmas / (best * 1e-3);
        for (auto& e : ev) cudaEventDestroy(e);
        return OF_OK;
    } catch (const Error& e) {
        for (auto& x : ev) if (x) cudaEventDestroy(x);
        return e.code;
    } catch (...) {
        for (auto& x : ev) if (x) cudaEventDestroy(x);
        return unexpected_exception();
    }
}

}  // extern "C"
