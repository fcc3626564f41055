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

// e = eps_xc(rho) * rho and v = V_xc(rho) for the exchange (Slater) and PZ correlation.
__device__ __forceinline__ void lda_xc(double rho, double& e, double& v) {
    const double r = fmax(rho, OF_RHO_FLOOR);
    const double c = cbrt(r);                       // rho^{1/3} = u^{2/3}
    const double ex = -0.75 * OF_CX * c;            // eps_x
    const double vx = -OF_CX * c;                   // V_x
    const double rs = OF_RS0 / c;
    double ec, vc;
    if (rs >= 1.0) {
        const double sq = sqrt(rs);
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
    const double c = cbrt(rho);
    const double c2 = c * c;
    e = OF_CF * rho * c2;
    v = (5.0 / 3.0) * OF_CF * c2;
}

// Energy densities only (line-search evaluations)
__device__ __forceinline__ double tf_xc_energy(double rho) {
    double etf, vtf, exc, vxc;
    thomas_fermi(rho, etf, vtf);
    lda_xc(rho, exc, vxc);
    return etf + exc;
}

}  // namespace of
