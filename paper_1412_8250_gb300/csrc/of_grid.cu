// Grid handle, workspace, error reporting and the plain Laplacian entry point.
#include <atomic>
#include <cstdarg>
#include <exception>
#include <new>
#include <cstring>
#include <cmath>

#include "of_stencil.cuh"

namespace of {

unsigned long long g_launch_count = 0;
unsigned long long g_resource_count = 0;
thread_local double g_capture_bytes = 0.0;
thread_local bool g_capturing = false;
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

of_status unexpected_exception() {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return OF_ENOMEM;
    } catch (const std::exception& e) {
        set_error("unexpected host exception: %s", e.what());
        return OF_ECUDA;
    } catch (...) {
        set_error("unexpected host exception");
        return OF_ECUDA;
    }
}

int num_sms() {
    static std::atomic<int> cached{0};
    int v = cached.load(std::memory_order_relaxed);
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        v = v > 0 ? v : 1;
        cached.store(v, std::memory_order_relaxed);
    }
    return v;
}

void* ws(of_grid* g, int slot, size_t bytes) {
    Buffer& b = g->pool[slot];
    if (b.bytes < bytes) {
        if (b.ptr) {   // work queued on the handle's stream may still use the old buffer
            OF_CUDA(cudaStreamSynchronize(g->stream));
            OF_CUDA(cudaFree(b.ptr));
        }
        b.ptr = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.ptr, bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) for workspace slot %d: %s", bytes, slot, cudaGetErrorString(e));
            throw Error{OF_ENOMEM};
        }
        note_resource();
        b.bytes = bytes;
    }
    return b.ptr;
}

void fetch_scalars(of_grid* g, int first, int count, double* out) {
    OF_CUDA(cudaMemcpyAsync(g->s.host + first, g->s.scalars + first, sizeof(double) * count,
                            cudaMemcpyDeviceToHost, g->stream));
    OF_CUDA(cudaStreamSynchronize(g->stream));
    std::memcpy(out, g->s.host + first, sizeof(double) * count);
}

// Weights of Eq. FD:Laplacian:
//   w_0 = -(1/h^2) sum_{q=1}^N 1/q^2,  w_p = 2 (-1)^{p+1} (N!)^2 / (h^2 p^2 (N-p)! (N+p)!).
void fd_weights(int N, double h, double* w) {
    double s = 0.0;
    for (int q = 1; q <= N; ++q) s += 1.0 / ((double)q * q);
    w[0] = -s / (h * h);
    for (int p = 1; p <= N; ++p) {
        // (N!)^2 / ((N-p)! (N+p)!) = prod_{k=1}^{p} (N-p+k)/(N+k)
        double ratio = 1.0;
        for (int k = 1; k <= p; ++k) ratio *= (double)(N - p + k) / (double)(N + k);
        const double sgn = (p % 2 == 1) ? 1.0 : -1.0;
        w[p] = 2.0 * sgn * ratio / (h * h * p * p);
    }
    for (int p = N + 1; p <= OF_MAX_N; ++p) w[p] = 0.0;
}

// ---------------------------------------------------------------- plain Laplacian
template <typename T>
struct OpLap {
    const T* x;
    T* y;
    __device__ bool begin() { return true; }
    __device__ T load(long long i) const { return __ldg(x + i); }
    // two neighbours at an even index (FP32 fast path)
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ float2 load2(long long i) const { return __ldg(reinterpret_cast<const float2*>(x + i)); }
    __device__ void store(long long i, T, T lap) { y[i] = lap; }
    template <typename U = T, typename = std::enable_if_t<std::is_same<U, float>::value>>
    __device__ void store2(long long i, float2, float2 lap) { *reinterpret_cast<float2*>(y + i) = lap; }
    __device__ void end() {}
};

void laplacian(of_grid* g, of_dtype dt, const void* x, void* y) {
    if (dt == OF_F64) {
        launch_stencil<double, 2>(g, g->w64, OpLap<double>{(const double*)x, (double*)y});
    } else if (dt == OF_F32) {
        launch_stencil<float, 2>(g, g->w32, OpLap<float>{(const float*)x, (float*)y});
    } else {
        OF_REQUIRE(false, OF_EINVAL, "unknown dtype %d", (int)dt);
    }
}

}  // namespace of

using namespace of;

extern "C" {

const char* of_last_error(void) { return of::g_err; }

of_status of_grid_create(int n1, int n2, int n3, double L1, double L2, double L3,
                         int fd_half_order, void* stream, of_grid** out) {
    if (!out) { set_error("of_grid_create: out is NULL"); return OF_EINVAL; }
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1 || !(L1 > 0) || !(L2 > 0) || !(L3 > 0)) {
        set_error("of_grid_create: bad sizes n=(%d,%d,%d) L=(%g,%g,%g)", n1, n2, n3, L1, L2, L3);
        return OF_EINVAL;
    }
    if (fd_half_order != 1 && fd_half_order != 3 && fd_half_order != 6) {
        set_error("of_grid_create: fd_half_order %d not in {1, 3, 6}", fd_half_order);
        return OF_EINVAL;
    }
    of_grid* g = new (std::nothrow) of_grid();
    if (!g) { set_error("of_grid_create: host allocation failed"); return OF_ENOMEM; }
    try {
        g->d = Dims{n1, n2, n3, (long long)n1 * n2 * n3};
        g->L[0] = L1; g->L[1] = L2; g->L[2] = L3;
        const int n[3] = {n1, n2, n3};
        for (int a = 0; a < 3; ++a) g->h[a] = g->L[a] / n[a];
        g->dV = g->h[0] * g->h[1] * g->h[2];
        g->N = fd_half_order;
        g->w64.centre = 0.0;
        for (int a = 0; a < 3; ++a) {
            fd_weights(g->N, g->h[a], g->w64.w[a]);
            g->w64.centre += 2.0 * g->w64.w[a][0];
            for (int p = 0; p <= OF_MAX_N; ++p) g->w32.w[a][p] = (float)g->w64.w[a][p];
        }
        g->w32.centre = (float)g->w64.centre;
        g->stream = (cudaStream_t)stream;
        OF_CUDA(cudaGetDevice(&g->device));
        g->pool.resize(WS_NSLOTS);
        OF_CUDA(cudaMalloc(&g->s.partials, sizeof(double) * OF_RED_SLOTS * OF_MAX_RED_BLOCKS));
        OF_CUDA(cudaMalloc(&g->s.counter, sizeof(unsigned int) * 4));
        OF_CUDA(cudaMalloc(&g->s.scalars, sizeof(double) * OF_NSCALARS));
        for (int k = 0; k < 3; ++k) note_resource();
        // zeroed on the handle's stream and finished before the handle is returned: a plain
        // cudaMemset runs on the legacy default stream, which the non-blocking streams the
        // handle later runs on (stream pool, twin handle) do not wait for, and a reduction
        // that starts before its counter is zeroed miscounts its blocks
        OF_CUDA(cudaMemsetAsync(g->s.counter, 0, sizeof(unsigned int) * 4, g->stream));
        OF_CUDA(cudaMemsetAsync(g->s.scalars, 0, sizeof(double) * OF_NSCALARS, g->stream));
        OF_CUDA(cudaStreamSynchronize(g->stream));
        OF_CUDA(cudaMallocHost(&g->s.host, sizeof(double) * OF_NSCALARS));
        note_resource();
        *out = g;
        return OF_OK;
    } catch (const Error& e) {
        of_grid_destroy(g);
        return e.code;
    } catch (...) {
        of_grid_destroy(g);
        return unexpected_exception();
    }
}

of_status of_grid_destroy(of_grid* g) {
    if (!g) return OF_OK;
    if (g->worker) g->worker_destroy(g->worker);
    if (g->twin) of_grid_destroy(g->twin);
    if (g->twin_stream) cudaStreamDestroy(g->twin_stream);
    if (g->twin_in) cudaEventDestroy(g->twin_in);
    if (g->twin_out) cudaEventDestroy(g->twin_out);
    if (g->mg) mg_destroy(g->mg);
    if (g->graphs) destroy_graphs(g->graphs);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->cap_stream2) cudaStreamDestroy(g->cap_stream2);
    if (g->prof) {
        for (auto& r : g->prof->recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        for (auto e : g->prof->pool) cudaEventDestroy(e);
        delete g->prof;
    }
    for (auto& b : g->pool)
        if (b.ptr) cudaFree(b.ptr);
    if (g->s.partials) cudaFree(g->s.partials);
    if (g->s.counter) cudaFree(g->s.counter);
    if (g->s.scalars) cudaFree(g->s.scalars);
    if (g->s.host) cudaFreeHost(g->s.host);
    delete g;
    return OF_OK;
}

of_status of_laplacian_apply(of_grid* g, of_dtype dtype, const void* x, void* y) {
    if (!g || !x || !y) { set_error("of_laplacian_apply: null argument"); return OF_EINVAL; }
    if (x == y) { set_error("of_laplacian_apply: x and y must not alias"); return OF_EINVAL; }
    try {
        laplacian(g, dtype, x, y);
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

unsigned long long of_launch_count(void) {
    return __atomic_load_n(&of::g_launch_count, __ATOMIC_RELAXED);
}

unsigned long long of_resource_count(void) {
    return __atomic_load_n(&of::g_resource_count, __ATOMIC_RELAXED);
}

const char* of_kernel_class_name(int cls) {
    static const char* names[PC_N] = {"stencil_f64", "stencil_f32", "cg_stencil_f64",
                                      "cg_stencil_f32", "cocg_stencil_f64", "cocg_stencil_f32",
                                      "krylov_update", "mg_smooth", "mg_transfer",
                                      "line_energy", "ions", "other", "mg_pcg_pass_graph",
                                      "cg_cocg_iteration_pair_graph", "precond_net",
                                      "mg_cocg_pass_graph"};
    return (cls >= 0 && cls < PC_N) ? names[cls] : "";
}

of_status of_profile_enable(of_grid* g, int sample_every) {
    if (!g || sample_every < 0) { set_error("of_profile_enable: bad argument"); return OF_EINVAL; }
    try {
        if (g->twin) {
            const of_status st = of_profile_enable(g->twin, sample_every);
            if (st != OF_OK) return st;
        }
        if (!g->prof) g->prof = new Prof();
        Prof& p = *g->prof;
        OF_CUDA(cudaStreamSynchronize(g->stream));
        for (auto& r : p.recs) { p.pool.push_back(r.e0); p.pool.push_back(r.e1); }
        p.recs.clear();
        for (int c = 0; c < PC_N; ++c) { p.seen[c] = p.timed[c] = 0; p.ms[c] = p.bytes[c] = 0.0; }
        p.every = sample_every;
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

int of_profile_read(of_grid* g, of_kernel_stat* out, int max) {
    if (!g || !g->prof) return 0;
    try {
        // the timed launches of this handle and of its twin chain (whose solves ran beside it)
        std::vector<Prof*> ps;
        for (of_grid* h = g; h; h = h->twin) ps.push_back(h->prof);
        OF_CUDA(cudaStreamSynchronize(g->stream));
        for (Prof* pp : ps) {
            if (!pp) continue;
            for (auto& r : pp->recs) {
                float ms = 0.f;
                OF_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
                pp->timed[r.cls] += 1;
                pp->ms[r.cls] += ms;
                pp->bytes[r.cls] += r.bytes;
                pp->pool.push_back(r.e0);
                pp->pool.push_back(r.e1);
            }
            pp->recs.clear();
        }
        int k = 0;
        for (int c = 0; c < PC_N && k < max; ++c) {
            long long seen = 0, timed = 0;
            double ms = 0.0, bytes = 0.0;
            for (Prof* pp : ps) {
                if (!pp) continue;
                seen += pp->seen[c];
                timed += pp->timed[c];
                ms += pp->ms[c];
                bytes += pp->bytes[c];
            }
            if (seen == 0) continue;
            out[k].kernel_class = c;
            out[k].launches = seen;
            out[k].timed = timed;
            out[k].total_ms = ms;
            out[k].mean_ms = timed ? ms / timed : 0.0;
            out[k].bytes_per_launch = timed ? bytes / timed : 0.0;
            ++k;
        }
        return k;
    } catch (const Error&) {
        return -1;
    }
}

}  // extern "C"
