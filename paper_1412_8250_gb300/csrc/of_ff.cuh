// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers (about
// 48 significant bits), built from error-free transformations -- Knuth's TwoSum, Dekker's
// FastTwoSum and the FMA form of Dekker's TwoProduct -- so that a stencil sweep of an FP64
// field can run on the FP32 pipes, which GB300 has at 74x the FP64 rate.  Every operation is
// written with the round-to-nearest intrinsics, which the compiler neither contracts nor
// reorders.  The field is split into hi + lo pairs once, before the sweep: splitting each
// loaded value inside the sweep costs more FP64-pipe conversions than the sweep saves.
#pragma once

#include "of_stencil.cuh"

namespace of {

struct FF {
    float hi, lo;
};
struct FF2 {   // complex: real and imaginary parts
    FF x, y;
};

__device__ __forceinline__ FF ff_from(double v) {
    const float h = __double2float_rn(v);
    return FF{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double ff_to(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF2 ff_from(double2 v) { return FF2{ff_from(v.x), ff_from(v.y)}; }
__device__ __forceinline__ double2 ff_to(FF2 a) { return make_double2(ff_to(a.x), ff_to(a.y)); }

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (FastTwoSum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // the rounding error of p, exactly
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// the stencil kernels' value arithmetic (weights are FF too)
__device__ __forceinline__ FF vadd(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ FF vmul(FF w, FF a) { return ff_mul(w, a); }
__device__ __forceinline__ FF vfma(FF w, FF a, FF c) { return ff_add(c, ff_mul(w, a)); }
__device__ __forceinline__ FF2 vadd(FF2 a, FF2 b) { return FF2{ff_add(a.x, b.x), ff_add(a.y, b.y)}; }
__device__ __forceinline__ FF2 vmul(FF w, FF2 a) { return FF2{ff_mul(w, a.x), ff_mul(w, a.y)}; }
__device__ __forceinline__ FF2 vfma(FF w, FF2 a, FF2 c) { return FF2{vfma(w, a.x, c.x), vfma(w, a.y, c.y)}; }

template <> struct Real<FF> { using type = FF; };
template <> struct Real<FF2> { using type = FF; };

// The FD weights of a grid as double-float pairs
inline Weights<FF> ff_weights(const Weights<double>& w) {
    auto split = [](double v) {
        const float h = (float)v;
        return FF{h, (float)(v - (double)h)};
    };
    Weights<FF> r;
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p <= OF_MAX_N; ++p) r.w[a][p] = split(w.w[a][p]);
    r.centre = split(w.centre);
    return r;
}

// xf = x as hi + lo pairs
template <typename T64, typename TF>
__global__ void __launch_bounds__(256) k_ff_split(long long n, const T64* __restrict__ x, TF* __restrict__ xf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        xf[i] = ff_from(x[i]);
}

}  // namespace of
