// approx.cuh -- the hardware's single-instruction square root and reciprocal
// (PTX sqrt.approx.f32 and rcp.approx.f32, both on the XU), for terms whose
// result is only scaled by a later rounding: the Smagorinsky relaxation
// frequency, where an error of an ulp in omega moves a population by an ulp of
// omega (feq - f), far below the FP32 step's own rounding.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

__device__ __forceinline__ float approx_sqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float approx_rcp(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Smagorinsky relaxation frequency (SI section 1): from the contraction
// pp = Pi^neq : Pi^neq of the non-equilibrium second moment,
// tau_eff = (tau + sqrt(tau^2 + 18 (C_s Delta)^2 sqrt(2 pp) / rho)) / 2 and
// omega = 1 / tau_eff.  c18 = 18 (C_s Delta)^2, inv_rho = 1/rho.
__device__ __forceinline__ float smagorinsky_omega(float pp, float inv_rho, float tau,
                                                   float tau_sq, float c18) {
  const float qn = approx_sqrt(2.0f * pp);
  const float r = approx_sqrt(fmaf(c18 * qn, inv_rho, tau_sq));
  return 2.0f * approx_rcp(tau + r);
}

}  // namespace lbm
