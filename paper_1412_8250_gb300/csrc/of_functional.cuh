// Pointwise energy densities and potentials (Sec. 2 and Sec. 3.3.1), device side.
#pragma once

#include <cuda_runtime.h>

namespace of {

// C_F = (3/10)(3 pi^2)^{2/3}  (Eq. LR:KineticEnergy)
constexpr double OF_CF = 2.8712340001881915;
// (3/pi)^{1/3}, the exchange prefactor of V_x (Sec. 3.3.1); eps_x carries 3/4 of it
constexpr double OF_CX = 0.98474502184269654;
// (3/(4 pi))^{1/3}: r_s = OF_RS0 * rho^{-1/3}
constexpr double OF_RS0 = 0.62035049089940009;
constexpr double OF_RHO_FLOOR = 1e-24;   // xc terms use max(rho, floor)
constexpr double OF_U_FLOOR = 1e-12;     // negative powers of u use max(u, floor)

// Perdew-Zunger constants as printed in Sec. 2
constexpr double PZ_G1 = -0.1423, PZ_B1 = 1.0529, PZ_B2 = 0.3334;
constexpr double PZ_A1 = 0.0311, PZ_BB1 = -0.048, PZ_C1 = 0.002, PZ_D1 = -0.0116;

// rho^{-1/3} by Newton's method for f(t) = t^{-3} - rho, t <- t (4 - rho t^3) / 3, from a
// single-precision seed; the error squares each step (1e-7 -> 1e-14 -> rounding), so two
// FP64 steps reach full double accuracy at a fraction of the cost of a double cube root.
__device__ __forceinline__ double inv_cbrt(double rho) {
    double t = (double)rcbrtf((float)rho);
#pragma unroll
    for (int k = 0; k < 2; ++k) t = t * (4.0 - rho * t * t * t) * (1.0 / 3.0);
    return t;
}

// sqrt(x) = x / sqrt(x) with 1/sqrt(x) from Newton's method y <- y (3 - x y^2) / 2 on a
// single-precision seed (two FP64 steps)
__device__ __forceinline__ double sqrt_newton(double x) {
    double y = (double)rsqrtf((float)x);
#pragma unroll
    for (int k = 0; k < 2; ++k) y = y * (1.5 - 0.5 * x * y * y);
    return x * y;
}

// 1/x by Newton's method y <- y (2 - x y), written as e = 1 - x y, y <- y + y e, from a
// single-precision seed (two FP64 steps: 1e-7 -> 1e-14 -> rounding); x a normal float.
__device__ __forceinline__ double rcp_newton(double x) {
    double y = (double)__frcp_rn((float)x);
#pragma unroll
    for (int k = 0; k < 2; ++k) y = fma(y, fma(-x, y, 1.0), y);
    return y;
}

// e = eps_xc(rho) * rho and v = V_xc(rho) for the exchange (Slater) and PZ correlation.
__device__ __forceinline__ void lda_xc(double rho, double& e, double& v) {
    const double r = fmax(rho, OF_RHO_FLOOR);
    const double t = inv_cbrt(r);                   // rho^{-1/3}
    const double c = r * t * t;                     // rho^{1/3} = u^{2/3}
    const double ex = -0.75 * OF_CX * c;            // eps_x
    const double vx = -OF_CX * c;                   // V_x
    const double rs = OF_RS0 * t;
    double ec, vc;
    if (rs >= 1.0) {
        const double sq = sqrt_newton(rs);
        const double den = 1.0 + PZ_B1 * sq + PZ_B2 * rs;
        ec = PZ_G1 / den;
        vc = (PZ_G1 + (7.0 / 6.0) * PZ_G1 * PZ_B1 * sq + (4.0 / 3.0) * PZ_G1 * PZ_B2 * rs) / (den * den);
    } else {
        const double lr = log(rs);
        ec = PZ_A1 * lr + PZ_BB1 + PZ_C1 * rs * lr + PZ_D1 * rs;
        vc = (PZ_A1 + (2.0 / 3.0) * PZ_C1 * rs) * lr + (PZ_BB1 - PZ_A1 / 3.0) +
             (1.0 / 3.0) * (2.0 * PZ_D1 - PZ_C1) * rs;
    }
    e = (ex + ec) * r;
    v = vx + vc;
}

// Thomas-Fermi: energy density C_F rho^{5/3} and V_TF = (5/3) C_F rho^{2/3}
__device__ __forceinline__ void thomas_fermi(double rho, double& e, double& v) {
    if (!(rho > 1e-30)) { e = 0.0; v = 0.0; return; }   // below 1e-50 Ha per point
    const double t = inv_cbrt(rho);
    const double c = rho * t * t;                   // rho^{1/3}
    const double c2 = c * c;
    e = OF_CF * rho * c2;
    v = (5.0 / 3.0) * OF_CF * c2;
}

// Energy densities only (line-search evaluations): C_F rho^{5/3} + eps_xc(rho) rho, one
// reciprocal cube root shared by both terms.
__device__ __forceinline__ double tf_xc_energy(double rho) {
    const double r = fmax(rho, OF_RHO_FLOOR);
    const double t = inv_cbrt(r);
    const double c = r * t * t;                     // rho^{1/3}
    const double etf = rho > 0.0 ? OF_CF * rho * c * c : 0.0;
    const double rs = OF_RS0 * t;
    double ec;
    if (rs >= 1.0) {
        ec = PZ_G1 / (1.0 + PZ_B1 * sqrt_newton(rs) + PZ_B2 * rs);
    } else {
        const double lr = log(rs);
        ec = PZ_A1 * lr + PZ_BB1 + PZ_C1 * rs * lr + PZ_D1 * rs;
    }
    return etf + (-0.75 * OF_CX * c + ec) * r;
}

// Energy density and its derivative along the line (slope line search): e = C_F rho^{5/3} +
// eps_xc(rho) rho as in tf_xc_energy, v = dE/drho = V_TF + V_xc, one reciprocal cube root and
// one Newton reciprocal of the Perdew-Zunger denominator shared by both.
__device__ __forceinline__ void tf_xc_energy_slope(double rho, double& e, double& v) {
    const double r = fmax(rho, OF_RHO_FLOOR);
    const double t = inv_cbrt(r);
    const double c = r * t * t;                     // rho^{1/3}
    const double tf = rho > 0.0 ? OF_CF * c * c : 0.0;   // C_F rho^{2/3}
    const double rs = OF_RS0 * t;
    double ec, vc;
    if (rs >= 1.0) {
        const double sq = sqrt_newton(rs);
        const double inv = rcp_newton(1.0 + PZ_B1 * sq + PZ_B2 * rs);
        ec = PZ_G1 * inv;
        vc = (PZ_G1 + (7.0 / 6.0) * PZ_G1 * PZ_B1 * sq + (4.0 / 3.0) * PZ_G1 * PZ_B2 * rs) * inv * inv;
    } else {
        const double lr = log(rs);
        ec = PZ_A1 * lr + PZ_BB1 + PZ_C1 * rs * lr + PZ_D1 * rs;
        vc = (PZ_A1 + (2.0 / 3.0) * PZ_C1 * rs) * lr + (PZ_BB1 - PZ_A1 / 3.0) +
             (1.0 / 3.0) * (2.0 * PZ_D1 - PZ_C1) * rs;
    }
    e = tf * rho + (-0.75 * OF_CX * c + ec) * r;
    v = (5.0 / 3.0) * tf - OF_CX * c + vc;
}

}  // namespace of
