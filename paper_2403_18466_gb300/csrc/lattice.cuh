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

// ---- arithmetic with explicit rounding, for one node (float) or two nodes
// at once (float2: packed f32x2 instructions).  Every operation below is a
// single IEEE round-to-nearest operation whose form (separate multiply and
// add, or one fused multiply-add) is written out, so the two forms give the
// same result in every lane and no kernel depends on the compiler's choice of
// contractions.
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a - b, rounded once (as fma(b, -1, a))
__device__ __forceinline__ float v_sub(float a, float b) { return __fmaf_rn(b, -1.0f, a); }
__device__ __forceinline__ float v_splat(float a, float) { return a; }
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 v_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 v_splat(float a, float2) { return make_float2(a, a); }
// 1/x rounded to nearest (per lane)
__device__ __forceinline__ float v_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float2 v_rcp(float2 x) {
  return make_float2(__frcp_rn(x.x), __frcp_rn(x.y));
}
template <class T> __device__ __forceinline__ T v_c(float a) { return v_splat(a, T()); }

template <class T>
struct MomentsT {
  T drho;     // rho - 1
  T rho;
  T ux, uy;
  T inv_rho;  // 1/rho, rounded to nearest
};
using Moments = MomentsT<float>;

template <class T>
__device__ __forceinline__ MomentsT<T> node_moments(const T d[Q]) {
  MomentsT<T> m;
  m.drho = v_add(v_add(v_add(d[0], d[1]), v_add(d[2], d[3])),
                 v_add(v_add(v_add(d[4], d[5]), v_add(d[6], d[7])), d[8]));
  const T jx = v_add(v_add(v_sub(d[1], d[3]), v_sub(d[5], d[6])), v_sub(d[8], d[7]));
  const T jy = v_sub(v_add(v_sub(d[2], d[4]), v_add(d[5], d[6])), v_add(d[7], d[8]));
  m.rho = v_add(v_c<T>(1.0f), m.drho);
  m.inv_rho = v_rcp(m.rho);
  m.ux = v_mul(jx, m.inv_rho);
  m.uy = v_mul(jy, m.inv_rho);
  return m;
}

// c_i . u for direction i (compile-time i)
template <class T>
__device__ __forceinline__ T c_dot_u(int i, const MomentsT<T> &m) {
  const int ax = cx(i), ay = cy(i);
  if (ax == 0 && ay == 0) return v_c<T>(0.0f);
  if (ay == 0) return ax > 0 ? m.ux : v_mul(v_c<T>(-1.0f), m.ux);
  if (ax == 0) return ay > 0 ? m.uy : v_mul(v_c<T>(-1.0f), m.uy);
  if (ax > 0) return ay > 0 ? v_add(m.ux, m.uy) : v_sub(m.ux, m.uy);
  return ay > 0 ? v_sub(m.uy, m.ux) : v_mul(v_c<T>(-1.0f), v_add(m.ux, m.uy));
}

// Shifted equilibrium deq_i = feq_i - w_i, Eq. S4 with cs^2 = 1/3:
//   deq_i = w_i (drho + rho (cu (3 + 4.5 cu) - 1.5 |u|^2)),  cu = c_i . u.
template <class T>
__device__ __forceinline__ void shifted_feq(const MomentsT<T> &m, T deq[Q]) {
  const T usq15 = v_mul(v_c<T>(1.5f), v_fma(m.ux, m.ux, v_mul(m.uy, m.uy)));
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const T cu = c_dot_u(i, m);
    const T q = v_fma(cu, v_fma(cu, v_c<T>(4.5f), v_c<T>(3.0f)), v_mul(v_c<T>(-1.0f), usq15));
    deq[i] = v_mul(v_c<T>(wf(i)), v_fma(m.rho, q, m.drho));
  }
}

// BGK relaxation d_i + (deq_i - d_i)/tau, Eq. S3.
template <class T>
__device__ __forceinline__ T bgk_relax(T d, T deq, T omega) {
  return v_fma(omega, v_sub(deq, d), d);
}

// EDM forcing term f_ext_i = feq_i(rho, u + F/rho) - feq_i(rho, u)  (Eq. S5)
// for F = (fx, 0), written without the cancellation of two equilibria.  With
// a = F/rho (a = F (1/rho), the rounded reciprocal of the moments, so no
// kernel divides here), s = 2 u_x + a_x, A = fx s and B = fx u_y, and using
// (c.u_s)^2 - (c.u)^2 = (c.a)(c.(2u + a)), |u_s|^2 - |u|^2 = a.(2u + a),
// rho a = F and c_x^2 = 1:
//   c_x = 0:    f_ext_i = -1.5 w_i A
//   c_x = +-1:  f_ext_i = 3 w_i (E_cx + 3 c_x c_y B),  E_+ = A + fx, E_- = A - fx
// (one or two fused multiply-adds per population).  Called with fx = 0 on a
// lattice without forcing, where it adds zeros.
template <class T>
__device__ __forceinline__ void add_edm_force_x(const MomentsT<T> &m, T fx, T out[Q]) {
  const T ax = v_mul(fx, m.inv_rho);
  const T A = v_mul(fx, v_fma(v_c<T>(2.0f), m.ux, ax));
  const T B = v_mul(fx, m.uy);
  const T Ep = v_add(A, fx), Em = v_sub(A, fx);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float w = wf(i);
    if (cx(i) == 0) {
      out[i] = v_fma(v_c<T>(-1.5f * w), A, out[i]);
    } else {
      T e = cx(i) > 0 ? Ep : Em;
      if (cy(i) != 0) e = v_fma(v_c<T>(3.0f * (float)(cx(i) * cy(i))), B, e);
      out[i] = v_fma(v_c<T>(3.0f * w), e, out[i]);
    }
  }
}

// True when |u| >= 0.4 or u is not finite (for two nodes: either of them).
__device__ __forceinline__ bool is_unstable(const Moments &m) {
  const float usq = m.ux * m.ux + m.uy * m.uy;
  return !(usq < UNSTABLE_USQ);
}
__device__ __forceinline__ bool is_unstable(const MomentsT<float2> &m, bool act_x, bool act_y) {
  const float2 usq = v_fma(m.ux, m.ux, v_mul(m.uy, m.uy));
  return (act_x && !(usq.x < UNSTABLE_USQ)) || (act_y && !(usq.y < UNSTABLE_USQ));
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
