// Ion terms: charge density of the nuclei (Sec. 3.2), self energy, the overlap correction
// E_c^* and f^c (App. B) and the Hellmann-Feynman forces (Eq. Force:Nuclei).
//
// Each ion carries a Gaussian charge b_J(r) = -Z_J (2 pi s^2)^{-3/2} exp(-r^2/(2 s^2)),
// r <= r_c, whose potential is V_J(r) = -Z_J erf(r/(sqrt2 s))/r.  Work is organised as one
// CUDA block per (ion, z-plane of the ion's bounding box); the box is addressed with
// unwrapped grid indices, each of which is one periodic image of the ion (Sec. 4: indices
// outside the grid map to their periodic image).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "of_stencil.cuh"

namespace of {

struct AtomBox {
    double R[3];
    double Z;
    int lo[3];
    int len[3];
};

struct AtomSet {
    AtomBox* d_boxes;   // device
    int n_atoms;
    int max_planes;     // max box extent along z
    std::vector<AtomBox> h;
};

static AtomSet upload_atoms(of_grid* g, const of_system* sys) {
    OF_REQUIRE(sys && sys->n_atoms >= 1 && sys->R && sys->Z && sys->sigma > 0 && sys->rc > 0,
               OF_EINVAL, "invalid of_system");
    AtomSet a;
    a.n_atoms = sys->n_atoms;
    a.h.resize(a.n_atoms);
    a.max_planes = 0;
    for (int J = 0; J < a.n_atoms; ++J) {
        AtomBox& b = a.h[J];
        b.Z = sys->Z[J];
        OF_REQUIRE(std::isfinite(b.Z), OF_EINVAL, "ion %d has a non-finite charge", J);
        for (int c = 0; c < 3; ++c) {
            b.R[c] = sys->R[3 * J + c];
            OF_REQUIRE(std::isfinite(b.R[c]), OF_EINVAL, "ion %d has a non-finite position", J);
            const int lo = (int)std::ceil((b.R[c] - sys->rc) / g->h[c]);
            const int hi = (int)std::floor((b.R[c] + sys->rc) / g->h[c]);
            b.lo[c] = lo;
            b.len[c] = hi - lo + 1;
        }
        a.max_planes = std::max(a.max_planes, a.h[J].len[2]);
    }
    a.d_boxes = (AtomBox*)ws(g, WS_ATOM, sizeof(AtomBox) * a.n_atoms);
    OF_CUDA(cudaMemcpyAsync(a.d_boxes, a.h.data(), sizeof(AtomBox) * a.n_atoms,
                            cudaMemcpyHostToDevice, g->stream));
    return a;
}

struct Gauss {
    double sigma, rc, norm, inv2s2, erfscale, v0;
};

static Gauss gauss(const of_system* sys) {
    Gauss q;
    q.sigma = sys->sigma;
    q.rc = sys->rc;
    q.norm = std::pow(2.0 * M_PI * sys->sigma * sys->sigma, -1.5);
    q.inv2s2 = 1.0 / (2.0 * sys->sigma * sys->sigma);
    q.erfscale = 1.0 / (std::sqrt(2.0) * sys->sigma);
    q.v0 = std::sqrt(2.0 / M_PI) / sys->sigma;
    return q;
}

__device__ __forceinline__ double gauss_b(double r2, double Z, const Gauss& q) {
    return -Z * q.norm * exp(-r2 * q.inv2s2);
}
__device__ __forceinline__ double gauss_V(double r, double Z, const Gauss& q) {
    return r < 1e-12 ? -Z * q.v0 : -Z * erf(r * q.erfscale) / r;
}

// V_J(r) = -Z_J g(r^2) with g(s) = erf(a sqrt s) / sqrt s, a = 1 / (sqrt2 sigma): an entire
// function of s = r^2, the same for every ion.  The self-energy and force kernels evaluate it
// at every point of every ion's ball, where an FP64 sqrt, erf and division per point set their
// time; they take it instead from a table of degree-VT_D polynomials on n equal intervals of
// s in [0, r_c^2] (Chebyshev interpolation at VT_D + 1 nodes per interval, converted to
// monomials in the interval's local variable x in [-1, 1]).  The interpolation error is below
// 2 (w / 4)^9 / 9! max |g^(9)| for an interval of width w in s, and |g^(k)| <= 2 a^(2k+1) /
// (sqrt(pi) (2k + 1)); n = ceil(2 a^2 r_c^2) intervals (w a^2 <= 1/2) keep it near 3e-15 of
// g(0) (checked for sigma = 0.3 ... 1.5, r_c = 3 ... 12).  Beyond VT_MAX intervals the kernels
// evaluate erf directly.
constexpr int VT_MAX = 256;
constexpr int VT_D = 8;
struct VTable {
    double c[VT_MAX][VT_D + 1];
    double s_scale;   // n / r_c^2
    int n;            // intervals; 0: evaluate erf directly
};

static VTable vtable(const of_system* sys) {
    VTable t{};
    const double a = 1.0 / (std::sqrt(2.0) * sys->sigma);
    const double smax = sys->rc * sys->rc;
    const double want = std::ceil(2.0 * a * a * smax);
    if (!(want <= VT_MAX)) return t;   // n = 0
    const int n = std::max(16, (int)want);
    const double w = smax / n;
    t.n = n;
    t.s_scale = n / smax;
    auto g = [a](double sv) { const double r = std::sqrt(sv); return std::erf(a * r) / r; };
    constexpr int M = VT_D + 1;
    // monomial coefficients of the Chebyshev polynomials T_0 .. T_VT_D
    double T[M][M] = {};
    T[0][0] = 1.0;
    T[1][1] = 1.0;
    for (int k = 2; k < M; ++k)
        for (int j = 0; j < M; ++j)
            T[k][j] = (j > 0 ? 2.0 * T[k - 1][j - 1] : 0.0) - T[k - 2][j];
    for (int i = 0; i < n; ++i) {
        double f[M], ck[M];
        for (int j = 0; j < M; ++j) {
            const double x = std::cos(M_PI * (j + 0.5) / M);
            f[j] = g(w * (i + 0.5 * (x + 1.0)));   // nodes are interior: s > 0
        }
        for (int k = 0; k < M; ++k) {
            double sum = 0.0;
            for (int j = 0; j < M; ++j) sum += f[j] * std::cos(M_PI * k * (j + 0.5) / M);
            ck[k] = (k == 0 ? 1.0 : 2.0) * sum / M;
        }
        for (int j = 0; j < M; ++j) {
            double m = 0.0;
            for (int k = j; k < M; ++k) m += ck[k] * T[k][j];
            t.c[i][j] = m;
        }
    }
    return t;
}

// g(s) from the table (in shared memory); 0 <= s <= r_c^2
__device__ __forceinline__ double vt_g(const double (*c)[VT_D + 1], double s_scale, int n, double s) {
    const double u = s * s_scale;
    const int i = min((int)u, n - 1);
    const double x = 2.0 * (u - (double)i) - 1.0;
    const double* q = c[i];
    double p = q[VT_D];
#pragma unroll
    for (int k = VT_D - 1; k >= 0; --k) p = fma(p, x, q[k]);
    return p;
}

__device__ __forceinline__ void vt_load(const VTable& t, double (*c)[VT_D + 1]) {
    for (int e = threadIdx.x; e < t.n * (VT_D + 1); e += blockDim.x) (&c[0][0])[e] = (&t.c[0][0])[e];
}

// V_J(r) at r^2 = s: from the table, or directly when it has none
__device__ __forceinline__ double vt_V(const VTable& t, const double (*c)[VT_D + 1], double s, double Z,
                                       const Gauss& q) {
    return t.n ? -Z * vt_g(c, t.s_scale, t.n, s) : gauss_V(sqrt(s), Z, q);
}

// The Gaussian factorises: exp(-r^2 / 2s^2) = ex(dx) ey(dy) ez(dz).  A block (J, plane) takes
// ex and ey of its box columns and rows from shared memory (one exp each per block) instead of
// one exp per point; boxes wider than GX_MAX fall back to the direct form.
constexpr int GX_MAX = 512;

__device__ __forceinline__ void gauss_axis_tables(const AtomBox& B, double h1, double h2, const Gauss& q,
                                                  double* ex, double* ey) {
    if (B.len[0] > GX_MAX || B.len[1] > GX_MAX) return;
    for (int t = threadIdx.x; t < B.len[0]; t += blockDim.x) {
        const double dx = (B.lo[0] + t) * h1 - B.R[0];
        ex[t] = exp(-dx * dx * q.inv2s2);
    }
    for (int t = threadIdx.x; t < B.len[1]; t += blockDim.x) {
        const double dy = (B.lo[1] + t) * h2 - B.R[1];
        ey[t] = exp(-dy * dy * q.inv2s2);
    }
}

// Block (J, plane): reduce dV * sum b_J V_J over the plane for the self energy, and with b
// non-null scatter b_J into b (atomic: boxes of different ions overlap, so the summation order
// of b, and its last bits, vary from run to run; the gather below is the deterministic form).
__global__ void __launch_bounds__(256) k_pseudocharge(Dims d, double h1, double h2, double h3,
                                                      const AtomBox* boxes, Gauss q, double* b,
                                                      double* e_self_part, int max_planes, const VTable vt) {
    const int J = blockIdx.x, pl = blockIdx.y;
    const AtomBox B = boxes[J];
    __shared__ double ex[GX_MAX], ey[GX_MAX];
    __shared__ double vc[VT_MAX][VT_D + 1];
    const bool tables = B.len[0] <= GX_MAX && B.len[1] <= GX_MAX;
    if (pl < B.len[2]) {
        gauss_axis_tables(B, h1, h2, q, ex, ey);
        vt_load(vt, vc);
    }
    __syncthreads();
    double acc = 0.0;
    if (pl < B.len[2]) {
        const int k = B.lo[2] + pl;
        const double dz = k * h3 - B.R[2];
        const double cz = -B.Z * q.norm * exp(-dz * dz * q.inv2s2);
        const int kw = wrap_index(k, d.n3);
        const double rc2 = q.rc * q.rc;
        // a warp per box row, its lanes along the row: the wrapped x index advances by 32
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
        for (int jj = warp; jj < B.len[1]; jj += nwarps) {
            const int j = B.lo[1] + jj;
            const double dy = j * h2 - B.R[1];
            const long long row = (long long)d.n1 * (wrap_index(j, d.n2) + (long long)d.n2 * kw);
            int iw = wrap_index(B.lo[0] + lane, d.n1);
            for (int ii = lane; ii < B.len[0]; ii += 32) {
                const double dx = (B.lo[0] + ii) * h1 - B.R[0];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= rc2) {
                    const double bj = tables ? cz * (ex[ii] * ey[jj]) : gauss_b(r2, B.Z, q);
                    if (b) atomicAdd(b + row + iw, bj);
                    acc += bj * vt_V(vt, vc, r2, B.Z, q);
                }
                iw += 32;
                while (iw >= d.n1) iw -= d.n1;
            }
        }
    }
    acc = warp_sum(acc);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        e_self_part[(long long)J * max_planes + pl] = s;
    }
}

// ---- the nuclear charge in a fixed summation order
// One periodic image of an ion: the ion's unwrapped box restricted to the grid by the offset
// off = m n (grid points) along each axis; its points are the in-grid indices lo..hi, and the
// displacement of point i is (i + off) h - R, the same arithmetic as in the unwrapped box.
struct IonImage {
    double R[3];
    double Z;
    int off[3];
    int lo[3];
    int hi[3];
};

constexpr int GT = 8;          // tile edge (points) of the gather
constexpr int GCAP = 64;       // images whose tables a block holds at once

__device__ __forceinline__ bool tile_overlaps(const IonImage& m, int x0, int y0, int z0) {
    return m.lo[0] <= x0 + GT - 1 && m.hi[0] >= x0 && m.lo[1] <= y0 + GT - 1 && m.hi[1] >= y0 &&
           m.lo[2] <= z0 + GT - 1 && m.hi[2] >= z0;
}

// Block = one 8 x 8 x 8 tile of the grid (z-slab blockIdx.z): b at each point is the sum over
// the images that reach the tile, taken in image order (ion order, then image offsets), each
// contribution -Z norm exp(-dz^2/2s^2) (exp(-dx^2/2s^2) exp(-dy^2/2s^2)) within r_c as in the
// scatter; the images of the slab come from a list built on the host.  Every point is written
// once, and the order of its sum does not depend on scheduling.
__global__ void __launch_bounds__(256) k_pseudocharge_gather(Dims d, double h1, double h2, double h3,
                                                             const IonImage* __restrict__ img,
                                                             const int* __restrict__ slab_start,
                                                             const int* __restrict__ slab_img, Gauss q,
                                                             double* __restrict__ b) {
    const int x0 = blockIdx.x * GT, y0 = blockIdx.y * GT, z0 = blockIdx.z * GT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid & 7, ty = (tid >> 3) & 7, tz = tid >> 6;   // points (tx, ty, tz) and (tx, ty, tz + 4)
    __shared__ int pend[256];
    __shared__ int wcount[8];
    __shared__ int npend;
    __shared__ double ex[GCAP][GT], ey[GCAP][GT], ez[GCAP][GT];   // ez carries -Z norm
    const double rc2 = q.rc * q.rc;
    const int i = x0 + tx, j = y0 + ty;
    double acc[2] = {0.0, 0.0};
    const int first = slab_start[blockIdx.z], last = slab_start[blockIdx.z + 1];
    for (int base = first; base < last; base += 256) {
        // the slab's images that reach this tile, compacted in order
        const int c = base + tid;
        const bool hit = c < last && tile_overlaps(img[slab_img[c]], x0, y0, z0);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) before += wcount[w];
            total += wcount[w];
        }
        if (hit) pend[before + __popc(bal & ((1u << lane) - 1u))] = slab_img[c];
        if (tid == 0) npend = total;
        __syncthreads();
        const int np = npend;
        for (int p0 = 0; p0 < np; p0 += GCAP) {
            const int cnt = min(GCAP, np - p0);
            // axis tables of this batch of images: one exp per (image, axis, tile coordinate)
            for (int e = tid; e < cnt * 3 * GT; e += 256) {
                const int m = e / (3 * GT), a = (e / GT) % 3, t = e % GT;
                const IonImage& I = img[pend[p0 + m]];
                const double hh = a == 0 ? h1 : (a == 1 ? h2 : h3);
                const int o = a == 0 ? x0 : (a == 1 ? y0 : z0);
                const double dv = (o + t + I.off[a]) * hh - I.R[a];
                const double ev = exp(-dv * dv * q.inv2s2);
                if (a == 0) ex[m][t] = ev;
                else if (a == 1) ey[m][t] = ev;
                else ez[m][t] = -I.Z * q.norm * ev;
            }
            __syncthreads();
            for (int m = 0; m < cnt; ++m) {
                const IonImage& I = img[pend[p0 + m]];
                const double dx = (i + I.off[0]) * h1 - I.R[0];
                const double dy = (j + I.off[1]) * h2 - I.R[1];
                const double exy = ex[m][tx] * ey[m][ty];
                const double dxy2 = dx * dx + dy * dy;
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const int kz = tz + 4 * s2;
                    const double dz = (z0 + kz + I.off[2]) * h3 - I.R[2];
                    if (dxy2 + dz * dz <= rc2) acc[s2] += ez[m][kz] * exy;
                }
            }
            __syncthreads();
        }
    }
    if (i < d.n1 && j < d.n2) {
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int k = z0 + tz + 4 * s2;
            if (k < d.n3) b[(long long)i + (long long)d.n1 * (j + (long long)d.n2 * k)] = acc[s2];
        }
    }
}

// Periodic images of the ions (each ion's unwrapped box split by the grid period) and, per
// z-slab of GT planes, the images that reach it, in image order.
static void build_images(of_grid* g, const AtomSet& a, IonImage*& d_img, int*& d_start, int*& d_list,
                         int& nslab) {
    const int n[3] = {g->d.n1, g->d.n2, g->d.n3};
    auto floor_div = [](int x, int m) { return x >= 0 ? x / m : -((-x + m - 1) / m); };
    std::vector<IonImage> im;
    for (const AtomBox& B : a.h) {
        int mlo[3], mhi[3];
        for (int c = 0; c < 3; ++c) {
            mlo[c] = floor_div(B.lo[c], n[c]);
            mhi[c] = floor_div(B.lo[c] + B.len[c] - 1, n[c]);
        }
        for (int mz = mlo[2]; mz <= mhi[2]; ++mz)
            for (int my = mlo[1]; my <= mhi[1]; ++my)
                for (int mx = mlo[0]; mx <= mhi[0]; ++mx) {
                    IonImage I;
                    const int m[3] = {mx, my, mz};
                    for (int c = 0; c < 3; ++c) {
                        I.R[c] = B.R[c];
                        I.off[c] = m[c] * n[c];
                        I.lo[c] = std::max(0, B.lo[c] - I.off[c]);
                        I.hi[c] = std::min(n[c] - 1, B.lo[c] + B.len[c] - 1 - I.off[c]);
                    }
                    I.Z = B.Z;
                    if (I.lo[0] <= I.hi[0] && I.lo[1] <= I.hi[1] && I.lo[2] <= I.hi[2]) im.push_back(I);
                }
    }
    nslab = (n[2] + GT - 1) / GT;
    std::vector<int> start(nslab + 1, 0), list;
    for (int s = 0; s < nslab; ++s) {
        start[s] = (int)list.size();
        for (int k = 0; k < (int)im.size(); ++k)
            if (im[k].lo[2] <= s * GT + GT - 1 && im[k].hi[2] >= s * GT) list.push_back(k);
    }
    start[nslab] = (int)list.size();
    const size_t b_img = (sizeof(IonImage) * im.size() + 255) / 256 * 256;
    const size_t b_start = (sizeof(int) * start.size() + 255) / 256 * 256;
    char* base = (char*)ws(g, WS_IMG, b_img + b_start + sizeof(int) * std::max<size_t>(1, list.size()));
    d_img = (IonImage*)base;
    d_start = (int*)(base + b_img);
    d_list = (int*)(base + b_img + b_start);
    OF_CUDA(cudaMemcpyAsync(d_img, im.data(), sizeof(IonImage) * im.size(), cudaMemcpyHostToDevice, g->stream));
    OF_CUDA(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, g->stream));
    if (!list.empty())
        OF_CUDA(cudaMemcpyAsync(d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, g->stream));
    // the host vectors go out of scope: finish the copies first
    OF_CUDA(cudaStreamSynchronize(g->stream));
}

// Block (J, plane): dV * sum grad b_J (phi - V_J) over the plane, 3 components.
__global__ void __launch_bounds__(256) k_forces(Dims d, double h1, double h2, double h3,
                                                const AtomBox* boxes, Gauss q, const double* phi,
                                                double* part, int max_planes, const VTable vt) {
    const int J = blockIdx.x, pl = blockIdx.y;
    const AtomBox B = boxes[J];
    __shared__ double ex[GX_MAX], ey[GX_MAX];
    __shared__ double vc[VT_MAX][VT_D + 1];
    const bool tables = B.len[0] <= GX_MAX && B.len[1] <= GX_MAX;
    if (pl < B.len[2]) {
        gauss_axis_tables(B, h1, h2, q, ex, ey);
        vt_load(vt, vc);
    }
    __syncthreads();
    double f[3] = {0.0, 0.0, 0.0};
    if (pl < B.len[2]) {
        const int k = B.lo[2] + pl;
        const double dz = k * h3 - B.R[2];
        const double cz = -B.Z * q.norm * exp(-dz * dz * q.inv2s2);
        const int kw = wrap_index(k, d.n3);
        const double rc2 = q.rc * q.rc;
        const double inv_s2 = 2.0 * q.inv2s2;
        // a warp per box row, its lanes along the row: the wrapped x index advances by 32
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
        for (int jj = warp; jj < B.len[1]; jj += nwarps) {
            const int j = B.lo[1] + jj;
            const double dy = j * h2 - B.R[1];
            const long long row = (long long)d.n1 * (wrap_index(j, d.n2) + (long long)d.n2 * kw);
            int iw = wrap_index(B.lo[0] + lane, d.n1);
            for (int ii = lane; ii < B.len[0]; ii += 32) {
                const double dx = (B.lo[0] + ii) * h1 - B.R[0];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= rc2) {
                    const double bj = tables ? cz * (ex[ii] * ey[jj]) : gauss_b(r2, B.Z, q);
                    // grad b_J = -b_J (x - R_J) / sigma^2
                    const double w = -bj * inv_s2 * (phi[row + iw] - vt_V(vt, vc, r2, B.Z, q));
                    f[0] += w * dx;
                    f[1] += w * dy;
                    f[2] += w * dz;
                }
                iw += 32;
                while (iw >= d.n1) iw -= d.n1;
            }
        }
    }
    __shared__ double sh[8][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double s = warp_sum(f[c]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
        part[((long long)J * max_planes + pl) * 3 + threadIdx.x] = s;
    }
}

// out[J*stride + c] = scale * sum over planes of part[(J*max_planes + pl)*stride + c]
__global__ void k_sum_planes(int n_atoms, int max_planes, int stride, const double* part,
                             double scale, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_atoms * stride) return;
    const int J = t / stride, c = t - J * stride;
    double s = 0.0;
    for (int pl = 0; pl < max_planes; ++pl) s += part[((long long)J * max_planes + pl) * stride + c];
    out[t] = scale * s;
}

// E_c^* (per-ion halves) and f^c for Gaussian charges with point reference charges:
// E_c^* = 1/2 sum_I sum_{(J,T) != (I,0)} Z_I Z_J erfc(r/(2s))/r, f^c_I = -dE_c^*/dR_I.
// One block per ion I; its threads take the (J, image) pairs in a fixed stride and the block
// sums them in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_overlap(int M, const AtomBox* boxes, double L1, double L2,
                                                 double L3, double sigma, double cutoff, int t1,
                                                 int t2, int t3, double* e_part, double* fc) {
    const int I = blockIdx.x;
    const AtomBox A = boxes[I];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // e, f0, f1, f2
    const double inv2s = 1.0 / (2.0 * sigma), c2 = cutoff * cutoff;
    const double gp0 = 1.0 / (sigma * sqrt(M_PI));
    const int na = 2 * t1 + 1, nb = 2 * t2 + 1, nc = 2 * t3 + 1;
    const int nimg = na * nb * nc;
    const long long total = (long long)M * nimg;
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
        const int J = (int)(t / nimg);
        int rem = (int)(t - (long long)J * nimg);
        const int a = rem / (nb * nc) - t1;
        rem %= nb * nc;
        const int bb = rem / nc - t2, c = rem % nc - t3;
        if (J == I && a == 0 && bb == 0 && c == 0) continue;
        const AtomBox B = boxes[J];
        const double dx = A.R[0] - B.R[0] - a * L1;
        const double dy = A.R[1] - B.R[1] - bb * L2;
        const double dz = A.R[2] - B.R[2] - c * L3;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > c2) continue;
        const double r = sqrt(r2);
        const double ec = erfc(r * inv2s);
        acc[0] += 0.5 * A.Z * B.Z * ec / r;
        // g'(r) = -exp(-r^2/(4 s^2)) / (s sqrt(pi) r) - erfc(r/2s)/r^2
        const double gp = -exp(-r2 * inv2s * inv2s) * gp0 / r - ec / r2;
        const double w = -A.Z * B.Z * gp / r;
        acc[1] += w * dx;
        acc[2] += w * dy;
        acc[3] += w * dz;
    }
    __shared__ double sh[8][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum(acc[k]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        if (threadIdx.x == 0) e_part[I] = v;
        else fc[3 * I + threadIdx.x - 1] = v;
    }
}

// ---- E_c^* and f^c on the grid with Gaussian reference charges (App. B)
// Reference charges b~_J of width sigma_ref within rc_ref, with the sign of b_J, so that
// b~ - b is neutral; V_c solves -(1/4pi) L_h V_c = b~ - b, and
//   E_c^* = 1/2 int (b~ + b) V_c + 1/2 sum_J int b_J V_J - 1/2 sum_J int b~_J V~_J.
// f^c follows the expression printed after Eq. RepulsiveCorrection2:
//   f_J = 1/2 sum_J' int [ grad b~_J' (V_c - V~_J') + grad b_J' (V_c + V_J')
//                          + grad(V~_J' - V_J') (b~ + b) + b_J' grad V_J' - b~_J' grad V~_J' ].

// (1/r) dV/dr of V = -Z erf(r/(sqrt2 s))/r, so that grad V = g(r) (x - R); near r = 0 the
// series Z v0/(3 s^2) (1 - 3 r^2/(10 s^2)) avoids the cancellation of the two terms.
__device__ __forceinline__ double gauss_gradV_over_r(double r2, double Z, const Gauss& q) {
    const double x2 = r2 * q.inv2s2;   // (r / (sqrt2 s))^2
    if (x2 < 1e-4) return Z * q.v0 * (2.0 * q.inv2s2) / 3.0 * (1.0 - 0.6 * x2);
    const double r = sqrt(r2);
    return -Z * (q.v0 * exp(-x2) / r - erf(r * q.erfscale) / r2) / r;
}

// Block (J, plane) of the box of radius `cut` (>= rc, rc_ref): the three components of the
// integrand above summed over the plane (the factor dV/2 is applied by k_sum_planes).
// Vc: the grid potential with its constant; bsum: b~ + b.
__global__ void __launch_bounds__(256) k_overlap_grid_forces(Dims d, double h1, double h2, double h3,
                                                             const AtomBox* boxes, Gauss q, Gauss qt,
                                                             double cut, const double* Vc,
                                                             const double* bsum, double* part,
                                                             int max_planes) {
    const int J = blockIdx.x, pl = blockIdx.y;
    const AtomBox B = boxes[J];
    double f[3] = {0.0, 0.0, 0.0};
    if (pl < B.len[2]) {
        const int k = B.lo[2] + pl;
        const double dz = k * h3 - B.R[2];
        const int kw = wrap_index(k, d.n3);
        const int nxy = B.len[0] * B.len[1];
        const double cut2 = cut * cut, rc2 = q.rc * q.rc, rct2 = qt.rc * qt.rc;
        const double inv_s2 = 2.0 * q.inv2s2, inv_st2 = 2.0 * qt.inv2s2;
        for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
            const int jj = t / B.len[0];
            const int i = B.lo[0] + (t - jj * B.len[0]);
            const int j = B.lo[1] + jj;
            const double dx = i * h1 - B.R[0], dy = j * h2 - B.R[1];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > cut2) continue;
            const long long idx = wrap_index(i, d.n1) +
                                  (long long)d.n1 * (wrap_index(j, d.n2) + (long long)d.n2 * kw);
            const double g = gauss_gradV_over_r(r2, B.Z, q);
            const double gt = gauss_gradV_over_r(r2, B.Z, qt);
            // grad (V~_J - V_J) (b~ + b)
            double w = (gt - g) * bsum[idx];
            if (r2 <= rc2 || r2 <= rct2) {
                const double vc = Vc[idx];
                const double r = sqrt(r2);
                if (r2 <= rc2) {   // grad b_J (V_c + V_J) + b_J grad V_J, grad b_J = -b_J (x-R)/s^2
                    const double bj = gauss_b(r2, B.Z, q);
                    w += -bj * inv_s2 * (vc + gauss_V(r, B.Z, q)) + bj * g;
                }
                if (r2 <= rct2) {  // grad b~_J (V_c - V~_J) - b~_J grad V~_J
                    const double btj = gauss_b(r2, B.Z, qt);
                    w += -btj * inv_st2 * (vc - gauss_V(r, B.Z, qt)) - btj * gt;
                }
            }
            f[0] += w * dx;
            f[1] += w * dy;
            f[2] += w * dz;
        }
    }
    __shared__ double sh[8][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double s = warp_sum(f[c]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
        part[((long long)J * max_planes + pl) * 3 + threadIdx.x] = s;
    }
}

// out = alpha x + beta y
__global__ void k_axpby_fields(long long n, double alpha, const double* x, double beta,
                               const double* y, double* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = alpha * x[i] + beta * y[i];
}

// x += c
__global__ void k_add_constant(long long n, double* x, double c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] += c;
}

// ---- b_J = -(1/4pi) L_h V_J (the paper's construction from the potential, Sec. 4)
// V_J sampled on the ion's ball box widened by N points each way: box point (i, j, k), with
// i = 0 .. n[0] - 1 standing for grid index lo[0] - N + i (unwrapped)
struct WideBox {
    int lo[3];   // unwrapped grid index of the ball box's first point
    int n[3];    // widened box extents (ball box + 2N)
    double R[3];
    double Z;
};

__global__ void k_sample_V(WideBox B, int N, double h1, double h2, double h3, Gauss q, double* V) {
    const long long nb = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nb;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % B.n[0]), j = (int)((t / B.n[0]) % B.n[1]),
                  k = (int)(t / ((long long)B.n[0] * B.n[1]));
        const double dx = (B.lo[0] - N + i) * h1 - B.R[0], dy = (B.lo[1] - N + j) * h2 - B.R[1],
                     dz = (B.lo[2] - N + k) * h3 - B.R[2];
        V[t] = gauss_V(sqrt(dx * dx + dy * dy + dz * dz), B.Z, q);
    }
}

// For the ball points of the box: b_J = -(1/4pi) (L_h V_J) from the samples (every tap inside
// the widened box), scattered into b (atomic: boxes overlap); sums b_J V_J for the self energy
template <int N>
__global__ void __launch_bounds__(256) k_box_lap(WideBox B, Dims d, double h1, double h2, double h3,
                                                 Weights<double> Wt, double rc, const double* V,
                                                 double* b, RedCtx rc_out) {
    double acc[1] = {0.0};
    const int m0 = B.n[0] - 2 * N, m1 = B.n[1] - 2 * N, m2 = B.n[2] - 2 * N;
    const long long nin = (long long)m0 * m1 * m2;
    const long long sy = B.n[0], sz = (long long)B.n[0] * B.n[1];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nin;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % m0), j = (int)((t / m0) % m1), k = (int)(t / ((long long)m0 * m1));
        const int gi = B.lo[0] + i, gj = B.lo[1] + j, gk = B.lo[2] + k;
        const double dx = gi * h1 - B.R[0], dy = gj * h2 - B.R[1], dz = gk * h3 - B.R[2];
        if (dx * dx + dy * dy + dz * dz > rc * rc) continue;
        const long long c = (i + N) + (j + N) * sy + (k + N) * sz;
        double lap = Wt.centre * V[c];
        for (int p = 1; p <= N; ++p)
            lap += Wt.w[0][p] * (V[c + p] + V[c - p]) + Wt.w[1][p] * (V[c + p * sy] + V[c - p * sy]) +
                   Wt.w[2][p] * (V[c + p * sz] + V[c - p * sz]);
        const double bj = -lap / (4.0 * M_PI);
        const long long idx = wrap_index(gi, d.n1) +
                              (long long)d.n1 * (wrap_index(gj, d.n2) + (long long)d.n2 * wrap_index(gk, d.n3));
        atomicAdd(b + idx, bj);
        acc[0] += bj * V[c];
    }
    grid_reduce<1>(acc, rc_out.partials, rc_out.counter, rc_out.out);
}

static void pseudocharge_fd(of_grid* g, const of_system* sys, double* b, double* e_self) {
    AtomSet a = upload_atoms(g, sys);
    Gauss q = gauss(sys);
    const int N = g->N;
    size_t max_box = 0;
    std::vector<WideBox> boxes(a.n_atoms);
    for (int J = 0; J < a.n_atoms; ++J) {
        WideBox& w = boxes[J];
        for (int c = 0; c < 3; ++c) {
            w.lo[c] = a.h[J].lo[c];
            w.n[c] = a.h[J].len[c] + 2 * N;
            w.R[c] = a.h[J].R[c];
        }
        w.Z = a.h[J].Z;
        max_box = std::max(max_box, (size_t)w.n[0] * w.n[1] * w.n[2]);
    }
    double* V = (double*)ws(g, WS_ATOMBOX, sizeof(double) * max_box);
    double* per_atom = (double*)ws(g, WS_S15, sizeof(double) * ((size_t)a.n_atoms + 8));
    OF_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * g->d.n, g->stream));
    for (int J = 0; J < a.n_atoms; ++J) {   // one ion at a time through the shared box buffer
        const WideBox& w = boxes[J];
        const long long nb = (long long)w.n[0] * w.n[1] * w.n[2];
        launch(k_sample_V, red_blocks(nb, 1024), 256, g->stream, w, N, g->h[0], g->h[1], g->h[2], q, V);
        const long long nin = (long long)a.h[J].len[0] * a.h[J].len[1] * a.h[J].len[2];
        RedCtx rc{g->s.partials, g->s.counter, per_atom + J};
        const unsigned nbl = (unsigned)red_blocks(nin, 1024);
        switch (N) {
            case 1: launch(k_box_lap<1>, nbl, 256, g->stream, w, g->d, g->h[0], g->h[1], g->h[2], g->w64, sys->rc, (const double*)V, b, rc); break;
            case 3: launch(k_box_lap<3>, nbl, 256, g->stream, w, g->d, g->h[0], g->h[1], g->h[2], g->w64, sys->rc, (const double*)V, b, rc); break;
            default: launch(k_box_lap<6>, nbl, 256, g->stream, w, g->d, g->h[0], g->h[1], g->h[2], g->w64, sys->rc, (const double*)V, b, rc); break;
        }
        OF_LAUNCH_CHECK();
    }
    if (e_self) {
        launch(k_sum_product, 1, 256, g->stream, (long long)a.n_atoms, (const double*)per_atom,
               (const double*)nullptr, red_ctx(g, 119));
        OF_LAUNCH_CHECK();
        fetch_scalars(g, 119, 1, e_self);
        *e_self *= -0.5 * g->dV;
    }
}

static void pseudocharge_impl(of_grid* g, const of_system* sys, double* b, double* e_self) {
    if (sys && sys->b_from_potential) return pseudocharge_fd(g, sys, b, e_self);
    AtomSet a = upload_atoms(g, sys);
    Gauss q = gauss(sys);
    IonImage* img = nullptr;
    int *start = nullptr, *list = nullptr, nslab = 0;
    build_images(g, a, img, start, list, nslab);
    launch(k_pseudocharge_gather, dim3((g->d.n1 + GT - 1) / GT, (g->d.n2 + GT - 1) / GT, nslab), 256,
           g->stream, g->d, g->h[0], g->h[1], g->h[2], (const IonImage*)img, (const int*)start,
           (const int*)list, q, b);
    OF_LAUNCH_CHECK();
    if (e_self) {
        const size_t nparts = (size_t)a.n_atoms * a.max_planes;
        double* part = (double*)ws(g, WS_S15, sizeof(double) * (nparts + a.n_atoms + 8));
        OF_CUDA(cudaMemsetAsync(part, 0, sizeof(double) * nparts, g->stream));
        launch(k_pseudocharge, dim3(a.n_atoms, a.max_planes), 256, g->stream, g->d, g->h[0], g->h[1],
               g->h[2], a.d_boxes, q, (double*)nullptr, part, a.max_planes, vtable(sys));
        OF_LAUNCH_CHECK();
        double* per_atom = part + nparts;
        launch(k_sum_planes, (a.n_atoms + 127) / 128, 128, g->stream, a.n_atoms, a.max_planes, 1,
                                                                    part, -0.5 * g->dV, per_atom);
        launch(k_sum_product, 1, 256, g->stream, a.n_atoms, per_atom, nullptr, red_ctx(g, 119));
        OF_LAUNCH_CHECK();
        fetch_scalars(g, 119, 1, e_self);
    }
}

// sum over the ions and their periodic images of (V~_J - V_J)(x0), terms beyond `cut` dropped
static double potential_difference_at(const double x0[3], const of_system* sys, const double L[3],
                                      double cut) {
    const double es = 1.0 / (std::sqrt(2.0) * sys->sigma), est = 1.0 / (std::sqrt(2.0) * sys->sigma_ref);
    int reps[3];
    for (int c = 0; c < 3; ++c) reps[c] = (int)std::ceil(cut / L[c]) + 1;
    double s = 0.0;
    for (int J = 0; J < sys->n_atoms; ++J)
        for (int a = -reps[0]; a <= reps[0]; ++a)
            for (int b = -reps[1]; b <= reps[1]; ++b)
                for (int c = -reps[2]; c <= reps[2]; ++c) {
                    const double dx = x0[0] - sys->R[3 * J] - a * L[0];
                    const double dy = x0[1] - sys->R[3 * J + 1] - b * L[1];
                    const double dz = x0[2] - sys->R[3 * J + 2] - c * L[2];
                    const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
                    if (r > cut) continue;
                    // V~_J - V_J = -Z (erf(r e~) - erf(r e)) / r, limit -Z (2/sqrt pi)(e~ - e)
                    s += r < 1e-12 ? -sys->Z[J] * 2.0 / std::sqrt(M_PI) * (est - es)
                                   : -sys->Z[J] * (std::erf(r * est) - std::erf(r * es)) / r;
                }
    return s;
}

// E_c^* and f^c of App. B on the grid (the comment above k_overlap_grid_forces)
static void overlap_correction_grid(of_grid* g, const of_system* sys, double* e_c, double* fc_host) {
    OF_REQUIRE(sys->rc_ref > 0 && !sys->b_from_potential, OF_EINVAL,
               "overlap correction on the grid: needs rc_ref > 0 and b_from_potential = 0");
    const long long n = g->d.n;
    const int nb = red_blocks(n, 256 * 4);
    double* f = (double*)ws(g, WS_OVL, sizeof(double) * 4 * (size_t)n);
    double *b = f, *bt = f + n, *rho = f + 2 * n, *Vc = f + 3 * n;
    of_system sb = *sys;   // the ions' charges as sampled from their closed form
    sb.b_from_potential = 0;
    of_system st = sb;     // the reference charges
    st.sigma = sys->sigma_ref;
    st.rc = sys->rc_ref;
    double self_b = 0.0, self_bt = 0.0;   // -1/2 sum_J int b_J V_J, and for b~
    pseudocharge_impl(g, &sb, b, &self_b);
    pseudocharge_impl(g, &st, bt, &self_bt);
    launch(k_axpby_fields, nb, 256, g->stream, n, 1.0, (const double*)bt, -1.0, (const double*)b, rho);
    OF_LAUNCH_CHECK();
    OF_CUDA(cudaMemsetAsync(Vc, 0, sizeof(double) * n, g->stream));
    KrylovOpts ko = krylov_opts(nullptr);
    ko.precision = OF_F32;   // FP32 multigrid passes refined in FP64
    ko.tol = 1e-12;
    const of_status ps = poisson(g, rho, Vc, ko, nullptr);
    OF_REQUIRE(ps == OF_OK, ps, "overlap correction on the grid: Poisson solve for V_c failed");
    // the constant of V_c: its value at the grid point x = 0 is the lattice sum of V~_J - V_J
    const double cut = 12.0 * std::max(sys->sigma, sys->sigma_ref);
    const double x0[3] = {0.0, 0.0, 0.0};
    const double s0 = potential_difference_at(x0, sys, g->L, cut);
    double v00 = 0.0;
    OF_CUDA(cudaMemcpyAsync(&v00, Vc, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    OF_CUDA(cudaStreamSynchronize(g->stream));
    const double c = s0 - v00;
    // b~ + b into rho
    launch(k_axpby_fields, nb, 256, g->stream, n, 1.0, (const double*)bt, 1.0, (const double*)b, rho);
    launch(k_add_constant, nb, 256, g->stream, n, Vc, c);
    OF_LAUNCH_CHECK();
    if (e_c) {
        launch(k_sum_product, nb, 256, g->stream, n, (const double*)rho, (const double*)Vc,
               red_ctx(g, 117));
        OF_LAUNCH_CHECK();
        double sv = 0.0;
        fetch_scalars(g, 117, 1, &sv);
        *e_c = 0.5 * g->dV * sv - self_b + self_bt;
    }
    if (fc_host) {
        of_system sc = sb;   // boxes of radius cut around each ion
        sc.rc = std::max(cut, std::max(sys->rc, sys->rc_ref));
        AtomSet a = upload_atoms(g, &sc);
        const int M = a.n_atoms;
        const size_t nparts = (size_t)M * a.max_planes * 3;
        double* part = (double*)ws(g, WS_OVLP, sizeof(double) * (nparts + 3 * (size_t)M + 8));
        double* per_atom = part + nparts;
        launch(k_overlap_grid_forces, dim3(M, a.max_planes), 256, g->stream, g->d, g->h[0], g->h[1],
               g->h[2], (const AtomBox*)a.d_boxes, gauss(&sb), gauss(&st), sc.rc,
               (const double*)Vc, (const double*)rho, part, a.max_planes);
        launch(k_sum_planes, (3 * M + 127) / 128, 128, g->stream, M, a.max_planes, 3,
               (const double*)part, 0.5 * g->dV, per_atom);
        OF_LAUNCH_CHECK();
        OF_CUDA(cudaMemcpyAsync(fc_host, per_atom, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost,
                                g->stream));
        OF_CUDA(cudaStreamSynchronize(g->stream));
    }
}

// E_c^* and f^c into host outputs (either may be null)
void overlap_correction(of_grid* g, const of_system* sys, double* e_c, double* fc_host) {
    if (sys && sys->sigma_ref > 0.0) return overlap_correction_grid(g, sys, e_c, fc_host);
    AtomSet a = upload_atoms(g, sys);
    const int M = a.n_atoms;
    const double cutoff = 14.0 * sys->sigma;
    const int t1 = (int)std::ceil(cutoff / g->L[0]) + 1;
    const int t2 = (int)std::ceil(cutoff / g->L[1]) + 1;
    const int t3 = (int)std::ceil(cutoff / g->L[2]) + 1;
    double* buf = (double*)ws(g, WS_S14, sizeof(double) * (4 * (size_t)M + 8));
    launch(k_overlap, M, 256, g->stream, M, a.d_boxes, g->L[0], g->L[1], g->L[2], sys->sigma,
           cutoff, t1, t2, t3, buf, buf + M);
    OF_LAUNCH_CHECK();
    if (e_c) {
        launch(k_sum_product, 1, 256, g->stream, M, buf, nullptr, red_ctx(g, 118));
        OF_LAUNCH_CHECK();
        fetch_scalars(g, 118, 1, e_c);
    }
    if (fc_host) {
        OF_CUDA(cudaMemcpyAsync(fc_host, buf + M, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost,
                                g->stream));
        OF_CUDA(cudaStreamSynchronize(g->stream));
    }
}

void pseudocharge(of_grid* g, const of_system* sys, double* b, double* e_self) {
    pseudocharge_impl(g, sys, b, e_self);
}

void forces(of_grid* g, const of_system* sys, const double* phi, double* F) {
    OF_REQUIRE(sys && sys->n_atoms >= 1, OF_EINVAL, "invalid of_system");
    std::vector<double> fc(3 * (size_t)sys->n_atoms);
    // f^c on the grid samples charges and solves for V_c in this handle's scratch (the ion
    // boxes and partial sums below reuse it), so it goes first; the closed form goes last
    const bool fc_on_grid = sys->sigma_ref > 0.0;
    if (fc_on_grid) overlap_correction(g, sys, nullptr, fc.data());   // synchronises the stream
    AtomSet a = upload_atoms(g, sys);
    Gauss q = gauss(sys);
    const int M = a.n_atoms;
    const size_t nparts = (size_t)M * a.max_planes * 3;
    double* part = (double*)ws(g, WS_S15, sizeof(double) * (nparts + 3 * (size_t)M + 8));
    double* per_atom = part + nparts;
    launch(k_forces, dim3(M, a.max_planes), 256, g->stream, g->d, g->h[0], g->h[1], g->h[2],
                                                         a.d_boxes, q, phi, part, a.max_planes, vtable(sys));
    OF_LAUNCH_CHECK();
    launch(k_sum_planes, (3 * M + 127) / 128, 128, g->stream, M, a.max_planes, 3, part, g->dV,
                                                            per_atom);
    OF_LAUNCH_CHECK();
    if (!fc_on_grid) overlap_correction(g, sys, nullptr, fc.data());   // synchronises the stream
    OF_CUDA(cudaMemcpyAsync(F, per_atom, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, g->stream));
    OF_CUDA(cudaStreamSynchronize(g->stream));
    for (size_t i = 0; i < fc.size(); ++i) F[i] += fc[i];
}

}  // namespace of

using namespace of;

extern "C" {

of_status of_pseudocharge(of_grid* g, const of_system* sys, double* b, double* e_self) {
    if (!g || !sys || !b) { set_error("of_pseudocharge: null argument"); return OF_EINVAL; }
    try {
        pseudocharge(g, sys, b, e_self);
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

of_status of_forces(of_grid* g, const of_system* sys, const double* u, const double* phi,
                    double* F) {
    (void)u;
    if (!g || !sys || !phi || !F) { set_error("of_forces: null argument"); return OF_EINVAL; }
    try {
        forces(g, sys, phi, F);
        return OF_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return unexpected_exception();
    }
}

}  // extern "C"
