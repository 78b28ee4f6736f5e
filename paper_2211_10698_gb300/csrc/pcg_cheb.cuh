// The Chebyshev preconditioner's step coefficients as a constant table (FP32 mixed solves).
#pragma once

#include "pcg_common.cuh"

namespace ccm {

// Coefficients of Chebyshev step j >= 1 for K~ z = r (Saad's recurrence on the eigenvalue
// interval of ChebCoef, z1 = r / theta): d_{j+1} = c1 d_j + c2 (r - K~ z_j),
// z_{j+1} = z_j + d_{j+1}, with d_1 = z_1, where with sigma1 = theta / delta,
//     rho_0 = 1 / sigma1,  rho_j = 1 / (2 sigma1 - rho_{j-1}),
//     c1 = rho_j rho_{j-1},  c2 = 2 rho_j / delta.
// They depend on j alone, so they are evaluated in FP64 by the compiler (each operation
// correctly rounded, as at run time) into a constant table: an FP64 division in every thread
// of every step would hold the narrow FP64 pipe for longer than the step's FP32 stencil.
constexpr int kChebSteps = 8;  // steps 1..7 (degree 8 at most)
constexpr double cheb_rho(int j) {
  const double sig1 = ChebCoef::theta / ChebCoef::delta;
  double rho = 1.0 / sig1;
  for (int q = 1; q <= j; ++q) rho = 1.0 / (2.0 * sig1 - rho);
  return rho;
}
constexpr float cheb_c1(int j) { return j < 1 ? 0.0f : (float)(cheb_rho(j) * cheb_rho(j - 1)); }
constexpr float cheb_c2(int j) { return j < 1 ? 0.0f : (float)(2.0 * cheb_rho(j) / ChebCoef::delta); }
static __constant__ float kChebC1[kChebSteps] = {cheb_c1(0), cheb_c1(1), cheb_c1(2), cheb_c1(3),
                                                 cheb_c1(4), cheb_c1(5), cheb_c1(6), cheb_c1(7)};
static __constant__ float kChebC2[kChebSteps] = {cheb_c2(0), cheb_c2(1), cheb_c2(2), cheb_c2(3),
                                                 cheb_c2(4), cheb_c2(5), cheb_c2(6), cheb_c2(7)};
__device__ __forceinline__ void cheb_step_coef(int j, float& c1, float& c2) {
  c1 = kChebC1[j];
  c2 = kChebC2[j];
}

}  // namespace ccm
