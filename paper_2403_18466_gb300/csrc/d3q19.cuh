// d3q19.cuh -- D3Q19 constants and per-node arithmetic (the paper's 3D setting).
//
// Velocity set and weights in the order of the paper's D3Q19 stencil table
// (SI section 1): 0 rest (1/3); 1..6 the axis neighbours (1/18):
// -x, -y, -z, +z, +y, +x; 7..18 the edge neighbours (1/36).
// State representation as for D2Q9: stored values are shifted by the weights,
// d_i = f_i - w_i, so rho - 1 = sum d_i and j = sum d_i c_i.
#pragma once
#include <cuda_runtime.h>

#include "approx.cuh"

namespace lbm {
namespace d3 {

constexpr int Q = 19;

__host__ __device__ constexpr int cx(int i) {
  return (i == 6 || i >= 15) ? 1 : ((i == 1 || (i >= 7 && i <= 10)) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 5 || i == 10 || i == 13 || i == 14 || i == 18)
             ? 1
             : ((i == 2 || i == 7 || i == 11 || i == 12 || i == 15) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 4 || i == 9 || i == 12 || i == 14 || i == 17)
             ? 1
             : ((i == 3 || i == 8 || i == 11 || i == 13 || i == 16) ? -1 : 0);
}
__host__ __device__ constexpr float wf(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// The paper's network: 19 -> 300 -> 300 -> 100 -> 19, LeakyReLU hidden layers.
constexpr int H1 = 300, H2 = 300, H3 = 100;
constexpr float LEAKY = 0.01f;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H1 * Q;
constexpr int OFF_W2 = OFF_B1 + H1;
constexpr int OFF_B2 = OFF_W2 + H2 * H1;
constexpr int OFF_W3 = OFF_B2 + H2;
constexpr int OFF_B3 = OFF_W3 + H3 * H2;
constexpr int OFF_W4 = OFF_B3 + H3;
constexpr int OFF_B4 = OFF_W4 + Q * H3;
constexpr int NPARAMS = OFF_B4 + Q;  // 128,319

constexpr float UNSTABLE_USQ = 0.16f;  // |u| >= 0.4 marks the run unstable

struct Moments {
  float drho, rho, ux, uy, uz;
  float inv_rho;  // 1/rho
};

__device__ __forceinline__ Moments node_moments(const float d[Q]) {
  Moments m;
  float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    s += d[i];
    if (cx(i)) jx += cx(i) > 0 ? d[i] : -d[i];
    if (cy(i)) jy += cy(i) > 0 ? d[i] : -d[i];
    if (cz(i)) jz += cz(i) > 0 ? d[i] : -d[i];
  }
  m.drho = s;
  m.rho = 1.0f + s;
  const float inv = 1.0f / m.rho;
  m.inv_rho = inv;
  m.ux = jx * inv;
  m.uy = jy * inv;
  m.uz = jz * inv;
  return m;
}

__device__ __forceinline__ float cdot(int i, float ax, float ay, float az) {
  return (float)cx(i) * ax + (float)cy(i) * ay + (float)cz(i) * az;
}

// Shifted equilibrium deq_i = feq_i - w_i (Eq. S4, cs^2 = 1/3).
__device__ __forceinline__ void shifted_feq(const Moments &m, float deq[Q]) {
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cu = cdot(i, m.ux, m.uy, m.uz);
    deq[i] = wf(i) * (m.drho + m.rho * (cu * (3.0f + 4.5f * cu) - usq15));
  }
}

// EDM forcing (Eq. S5) for a body force F: with a = F/rho and s = 2u + a,
// feq(rho, u + a) - feq(rho, u) = w_i [3 c.F + 4.5 (c.F)(c.s) - 1.5 F.s]
// (rho a = F), written without subtracting two equilibria.
__device__ __forceinline__ void add_edm_force(const Moments &m, float Fx, float Fy, float Fz,
                                              float out[Q]) {
  const float inv = 1.0f / m.rho;
  const float sx = 2.0f * m.ux + Fx * inv, sy = 2.0f * m.uy + Fy * inv,
              sz = 2.0f * m.uz + Fz * inv;
  const float Fs15 = 1.5f * (Fx * sx + Fy * sy + Fz * sz);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cF = cdot(i, Fx, Fy, Fz), cs = cdot(i, sx, sy, sz);
    out[i] += wf(i) * (cF * (3.0f + 4.5f * cs) - Fs15);
  }
}

// Smagorinsky tau_eff = (tau0 + sqrt(tau0^2 + 18 (C_s Delta)^2 Q / rho)) / 2 with
// Q = sqrt(2 Pi:Pi), Pi_ab = sum c_ia c_ib (f_i - feq_i) (SI section 1).
__device__ __forceinline__ float smag_omega(const float d[Q], const float deq[Q], float inv_rho,
                                            float tau0_sq, float tau0, float c18) {
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float n = d[i] - deq[i];
    if (cx(i)) pxx += n;
    if (cy(i)) pyy += n;
    if (cz(i)) pzz += n;
    if (cx(i) && cy(i)) pxy += cx(i) * cy(i) > 0 ? n : -n;
    if (cx(i) && cz(i)) pxz += cx(i) * cz(i) > 0 ? n : -n;
    if (cy(i) && cz(i)) pyz += cy(i) * cz(i) > 0 ? n : -n;
  }
  const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
  return smagorinsky_omega(pp, inv_rho, tau0, tau0_sq, c18);
}

__device__ __forceinline__ bool is_unstable(const Moments &m) {
  const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
  return !(usq < UNSTABLE_USQ);
}

// Conservation layer of the learned collision: ohat = o + k1 + k2 cx + k3 cy + k4 cz,
// k1 = -sum o / 19, k_a = -sum o c_a / 10.
__device__ __forceinline__ void project(float o[Q]) {
  float s = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    s += o[i];
    sx += (float)cx(i) * o[i];
    sy += (float)cy(i) * o[i];
    sz += (float)cz(i) * o[i];
  }
  const float k1 = -s * (1.0f / 19.0f), k2 = -sx * 0.1f, k3 = -sy * 0.1f, k4 = -sz * 0.1f;
#pragma unroll
  for (int i = 0; i < Q; ++i) o[i] += k1 + cdot(i, k2, k3, k4);
}

}  // namespace d3
}  // namespace lbm
