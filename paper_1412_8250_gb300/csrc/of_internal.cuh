// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/of.h"

#define OF_MAX_N 6
#define OF_RED_SLOTS 48          // scalars produced by one reduction kernel (max)
#define OF_MAX_RED_BLOCKS 4096   // partial sums per slot
#define OF_NSCALARS 384          // device solver scalars per grid handle

namespace of {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
struct Error {
    of_status code;
};
// Status for an exception other than Error that reached a C entry point (called inside the
// catch block): OF_ENOMEM for a failed host allocation, OF_ECUDA otherwise, with a message.
of_status unexpected_exception();

#define OF_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::of::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                   \
                            cudaGetErrorString(e_));                                     \
            throw ::of::Error{OF_ECUDA};                                                 \
        }                                                                                \
    } while (0)

#define OF_LAUNCH_CHECK() OF_CUDA(cudaGetLastError())

// Kernel launches by this library (process-wide), for the launch accounting of callers.
extern unsigned long long g_launch_count;

// Resources this library has created (process-wide): device and pinned host buffers, streams,
// events and executable graphs.  Every creation site calls note_resource() after it succeeds.
extern unsigned long long g_resource_count;
inline void note_resource() { __atomic_add_fetch(&g_resource_count, 1ull, __ATOMIC_RELAXED); }

// Every kernel of the library is launched through this wrapper (no dynamic shared memory).
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream,
                   Args&&... args) {
    kernel<<<grid, block, 0, stream>>>(std::forward<Args>(args)...);
    __atomic_add_fetch(&g_launch_count, 1ull, __ATOMIC_RELAXED);
    OF_CUDA(cudaGetLastError());
}

// Programmatic dependent launch, for the kernels of the solver loops: every kernel launched
// this way starts with pdl_enter(), which waits until the previous kernel of the stream has
// completed and its writes are visible; nothing a kernel reads from global memory is touched
// before it.  The launch of each kernel is prepared while the previous one runs.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    OF_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
    __atomic_add_fetch(&g_launch_count, 1ull, __ATOMIC_RELAXED);
}

// First statement of every kernel launched with launch_pdl (a no-op under a plain launch).
// No early trigger: the next kernel's blocks are released when this grid completes (released
// at the start, they sat resident beside this grid's blocks and slowed a 96^3 sweep from 5.8 to
// 8.1 us).
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Same, with `smem` bytes of dynamic shared memory (the caller raises the kernel's limit).
template <typename... KArgs, typename... Args>
inline void launch_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        cudaStream_t stream, Args&&... args) {
    kernel<<<grid, block, smem, stream>>>(std::forward<Args>(args)...);
    __atomic_add_fetch(&g_launch_count, 1ull, __ATOMIC_RELAXED);
    OF_CUDA(cudaGetLastError());
}

// Sampled per-class kernel timing with CUDA events on the launching stream.
enum ProfClass {
    PC_STENCIL_F64 = 0, PC_STENCIL_F32, PC_CG_F64, PC_CG_F32, PC_COCG_F64, PC_COCG_F32,
    PC_UPDATE, PC_MG_SMOOTH, PC_MG_TRANSFER, PC_LINE, PC_ATOMS, PC_OTHER, PC_PCG_GRAPH, PC_KRYLOV_GRAPH, PC_NET, PC_PCOCG_GRAPH, PC_N
};

// While a CUDA graph is being captured, ProfScope adds the algorithmic bytes of each captured
// launch here (per host thread), so the graph's replays can be reported with their traffic.
extern thread_local double g_capture_bytes;
extern thread_local bool g_capturing;
struct ProfRec {
    int cls;
    cudaEvent_t e0, e1;
    double bytes;
};
struct Prof {
    int every = 0;
    long long seen[PC_N] = {};
    long long timed[PC_N] = {};
    double ms[PC_N] = {};
    double bytes[PC_N] = {};
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    // sets the bytes of the latest timed launch of class cls not yet read (graph launches whose
    // traffic is known only after a later host read)
    void amend_last(int cls, double b) {
        for (auto it = recs.rbegin(); it != recs.rend(); ++it)
            if (it->cls == cls) {
                it->bytes = b;
                return;
            }
    }
    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            OF_CUDA(cudaEventCreate(&e));
            note_resource();
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
};

#define OF_REQUIRE(cond, code, ...)                                                      \
    do {                                                                                 \
        if (!(cond)) {                                                                   \
            ::of::set_error(__VA_ARGS__);                                                \
            throw ::of::Error{code};                                                     \
        }                                                                                \
    } while (0)

// ---------------------------------------------------------------- grid
struct Dims {
    int n1, n2, n3;
    long long n;
};

// Laplacian weights of Eq. FD:Laplacian per axis (index 0 = w_0), and their sum over axes of
// the two centre terms.
template <typename R>
struct Weights {
    R w[3][OF_MAX_N + 1];
    R centre;   // 2 (w_0^x + w_0^y + w_0^z)
};

// Device scratch for deterministic two-level reductions and solver scalars.
struct Scratch {
    double* partials = nullptr;       // [OF_RED_SLOTS * OF_MAX_RED_BLOCKS]
    unsigned int* counter = nullptr;  // block-arrival counter (one per reduction kernel)
    double* scalars = nullptr;        // general device scalars [OF_NSCALARS]
    double* host = nullptr;           // pinned host mirror [256]
};

// Growable pool of device buffers owned by a grid handle.
struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct MG;
void mg_destroy(MG* m);

}  // namespace of

struct of_grid {
    of::Dims d;
    double L[3];
    double h[3];
    double dV;
    int N;
    of::Weights<double> w64;
    of::Weights<float> w32;
    cudaStream_t stream;
    int device;
    of::Scratch s;
    std::vector<of::Buffer> pool;    // named workspace slots, see of::ws()
    of::MG* mg = nullptr;            // multigrid hierarchy (built on first use)
    of::Prof* prof = nullptr;        // kernel timing (of_profile_enable)
    cudaStream_t cap_stream = nullptr;   // private stream for CUDA-graph capture
    cudaStream_t cap_stream2 = nullptr;  // second capture stream (bodies of conditional nodes)
    // a second handle on the same grid (own workspace, graphs, stream) for a solve that runs
    // concurrently with one on this handle; created on first use
    of_grid* twin = nullptr;
    cudaStream_t twin_stream = nullptr;
    cudaEvent_t twin_in = nullptr, twin_out = nullptr;
    // host thread that runs the twin's half of paired solves (of_scf.cu), started with the
    // first pair and joined by worker_destroy when the handle is destroyed
    void* worker = nullptr;
    void (*worker_destroy)(void*) = nullptr;
    void* graphs = nullptr;              // cached CUDA graphs (of_krylov.cu)
    // the Krylov loops launch every iteration directly instead of capturing and caching CUDA
    // graphs (which create a capture stream and executable graphs)
    bool no_graphs = false;
};

namespace of {
struct ProfScope {
    Prof* p = nullptr;
    int cls;
    double bytes;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ended = false;
    ProfScope(of_grid* g, int cls_, double bytes_) : cls(cls_), bytes(bytes_), s(g->stream) {
        if (g_capturing) {
            g_capture_bytes += bytes;
            return;
        }
        p = g->prof;
        if (!p) return;
        if (p->every > 0 && (p->seen[cls] % p->every) == 0) {
            e0 = p->get();
            e1 = p->get();
            OF_CUDA(cudaEventRecord(e0, s));
        }
        p->seen[cls]++;
    }
    // ends the timed interval here (the record, with `bytes` as set by then, is kept at scope
    // exit): for a launch whose traffic is known only after a later host read
    void end_timing() {
        if (e0 && !ended) {
            cudaEventRecord(e1, s);
            ended = true;
        }
    }
    ~ProfScope() {
        if (e0) {
            if (!ended) cudaEventRecord(e1, s);
            p->recs.push_back(ProfRec{cls, e0, e1, bytes});
        }
    }
};
}  // namespace of

namespace of {

// Workspace slot ids (each a device buffer of at least the requested bytes).
enum Slot {
    WS_K0 = 0,   // Krylov vectors 0..7 (FP64 or FP32 / complex)
    WS_K1, WS_K2, WS_K3, WS_K4, WS_K5, WS_K6, WS_K7,
    WS_S0, WS_S1, WS_S2, WS_S3, WS_S4, WS_S5, WS_S6, WS_S7,   // SCF vectors
    WS_S8, WS_S9, WS_S10, WS_S11, WS_S12, WS_S13, WS_S14, WS_S15,
    WS_LR,       // kernel-solve warm starts
    WS_AND,      // Anderson history
    WS_ATOM,     // per-atom device data
    WS_ATOMBOX,  // one ion's widened box (pseudocharge from the potential)
    WS_OVL,      // reference charges, V_c and its right-hand side (overlap correction on the grid)
    WS_OVLP,     // per-(ion, plane) partial forces of that correction
    WS_MG,       // multigrid hierarchy
    WS_NLCGP,    // preconditioned NLCG: the gradient in FP32, its V-cycle, the FP64 direction
    WS_FGM,      // flexible GMRES: Arnoldi and preconditioned vectors
    WS_IMG,      // periodic images of the ions and their lists per z-slab (nuclear charge)
    WS_FF,       // a field split into double-float pairs (the mixed form's residual sweeps)
    WS_NSLOTS
};

void* ws(of_grid* g, int slot, size_t bytes);   // grow-only

// Weights w_0..w_N of Eq. FD:Laplacian for spacing h (w_p = 0 for N < p <= OF_MAX_N).
void fd_weights(int N, double h, double* w);

// Reduction bookkeeping: how many blocks a grid-sized kernel uses
inline int red_blocks(long long work_items, int per_block) {
    long long b = (work_items + per_block - 1) / per_block;
    if (b > OF_MAX_RED_BLOCKS) b = OF_MAX_RED_BLOCKS;
    if (b < 1) b = 1;
    return (int)b;
}

// Reads `count` device scalars (starting at index first of g->s.scalars) to host.
void fetch_scalars(of_grid* g, int first, int count, double* out);

// ----------------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic grid-wide sum of K per-thread values: block partials are stored in
// `partials[k * OF_MAX_RED_BLOCKS + block]`; the last block to finish adds them in block
// order and writes out[k].  Requires blockDim.x * blockDim.y * blockDim.z <= 1024 and a
// multiple of 32; every thread of the block must call it.
template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], double* partials,
                                            unsigned int* counter, double* out) {
    __shared__ double sh[32][K > 0 ? K : 1];
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = lane < nwarps ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            if (lane == 0) partials[k * OF_MAX_RED_BLOCKS + bid] = s;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned int)nblocks - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = tid; b < nblocks; b += nthreads)
            s += ((volatile double*)partials)[k * OF_MAX_RED_BLOCKS + b];
        s = warp_sum(s);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = lane < nwarps ? sh[lane][k] : 0.0;
            s = warp_sum(s);
            if (lane == 0) {
                out[k] = s;
                v[k] = s;   // thread 0 of the last block also gets the totals
            }
        }
    }
    if (tid == 0) *counter = 0u;
    return true;
}

// ------------------------------------------------------------- entry points of the units
void laplacian(of_grid* g, of_dtype dt, const void* x, void* y);

struct KrylovOpts {
    double tol;
    int max_iter;
    int precision;
    double inner_tol;
    int check_every;
    int no_multigrid;
    of_precond* precond;
    double theta;
};
KrylovOpts krylov_opts(const of_solve_opts* o);

// Poisson: -(1/4pi) L phi = rho (mean removed), phi mean-free on return.
of_status poisson(of_grid* g, const double* rho, double* phi, const KrylovOpts& o,
                  of_solve_info* info);
// Poisson with rhs given as rho = a*b (elementwise product of two fields), used by NLCG.
of_status poisson_product(of_grid* g, const double* a, const double* b, double* phi,
                          const KrylovOpts& o, of_solve_info* info);
// Shifted: (-(1/kf2) L + Q) W = P f, complex W interleaved.
of_status shifted(of_grid* g, const double* f, double2 P, double2 Q, double kf2, double2* W,
                  const KrylovOpts& o, of_solve_info* info);

}  // namespace of
