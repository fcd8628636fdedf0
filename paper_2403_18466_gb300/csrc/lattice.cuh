// lattice.cuh -- D2Q9 constants and per-node arithmetic shared by the kernels.
//
// State representation: populations are stored SHIFTED by their weights,
// d_i = f_i - w_i, so that near rest (rho ~ 1, |u| << 1) the stored values
// are small and FP32 keeps ~2 more decimal digits of the physically relevant
// deviation (shifted populations, Skordos 1993).  All arithmetic below is
// written in that form:
//   rho - 1 = sum_i d_i,            j = sum_i d_i c_i        (sum_i w_i c_i = 0)
//   feq_i - w_i = w_i [(rho - 1) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2)]  (Eq. S4)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int Q = 9;
// c_x, c_y and w of velocity i (folded to constants inside unrolled loops).
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr float wf(int i) {
  return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
constexpr int HIDDEN = 64;
constexpr int NPARAMS = HIDDEN * 9 + HIDDEN + HIDDEN * HIDDEN + HIDDEN + 9 * HIDDEN + 9;

// Offsets of the packed parameter vector: w1[64][9], b1, w2[64][64], b2, w3[9][64], b3.
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HIDDEN * 9;
constexpr int OFF_W2 = OFF_B1 + HIDDEN;
constexpr int OFF_B2 = OFF_W2 + HIDDEN * HIDDEN;
constexpr int OFF_W3 = OFF_B2 + HIDDEN;
constexpr int OFF_B3 = OFF_W3 + 9 * HIDDEN;

// |u|^2 at or above this marks the run unstable (|u| >= 0.4, or NaN).
constexpr float UNSTABLE_USQ = 0.16f;

struct Moments {
  float drho;  // rho - 1
  float rho;
  float ux, uy;
  float inv_rho;  // 1/rho, rounded to nearest
};

__device__ __forceinline__ Moments node_moments(const float d[Q]) {
  Moments m;
  m.drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
  const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
  const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
  m.rho = 1.0f + m.drho;
  const float inv = 1.0f / m.rho;
  m.inv_rho = inv;
  m.ux = jx * inv;
  m.uy = jy * inv;
  return m;
}

// Shifted equilibrium deq_i = feq_i - w_i, Eq. S4 with cs^2 = 1/3.
__device__ __forceinline__ void shifted_feq(const Moments &m, float deq[Q]) {
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cu = (float)cx(i) * m.ux + (float)cy(i) * m.uy;
    deq[i] = wf(i) * (m.drho + m.rho * (cu * (3.0f + 4.5f * cu) - usq15));
  }
}

// EDM forcing term f_ext_i = feq_i(rho, u + F/rho) - feq_i(rho, u)  (Eq. S5)
// for F = (fx, 0), written without the cancellation of two equilibria:
// with a = F/rho, (c.u_s)^2 - (c.u)^2 = (c.a)(c.(2u + a)) and
// |u_s|^2 - |u|^2 = a.(2u + a); rho a = F.  a = F (1/rho) with the rounded
// reciprocal of the moments, so no kernel divides here.
__device__ __forceinline__ void add_edm_force_x(const Moments &m, float fx, float out[Q]) {
  const float ax = fx * m.inv_rho;
  const float sx = 2.0f * m.ux + ax;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (cx(i) == 0) {
      out[i] -= wf(i) * fx * sx * 1.5f;  // only the -1.5 a.(2u+a) term survives
    } else {
      const float cs = (float)cx(i) * sx + (float)cy(i) * 2.0f * m.uy;
      out[i] += wf(i) * fx * ((float)cx(i) * (3.0f + 4.5f * cs) - 1.5f * sx);
    }
  }
}

// True when |u| >= 0.4 or u is not finite.
__device__ __forceinline__ bool is_unstable(const Moments &m) {
  const float usq = m.ux * m.ux + m.uy * m.uy;
  return !(usq < UNSTABLE_USQ);
}

// Sets the sticky flag if any calling lane is unstable: one read (and at most
// one atomic) per warp, so a blown-up state does not serialise on the flag.
// Call with the same control flow in all lanes that are active.
__device__ __forceinline__ void flag_unstable(bool bad, int *flag) {
  const unsigned mask = __ballot_sync(__activemask(), bad);
  if (mask && (threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
    if (*reinterpret_cast<volatile int *>(flag) == 0) atomicOr(flag, 1);
  }
}

__host__ __device__ __forceinline__ int wrap_index(int a, int n) {
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

}  // namespace lbm
