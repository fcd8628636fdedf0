// adjoint_tc.cu -- hand-written reverse mode of one unrolled learned-collision
// step (unrolled training, SI section 2) on the tensor cores: every product
// with a weight matrix, and every weight-gradient sum over nodes, is a tcgen05
// GEMM with BF16 operands and FP32 accumulation.  The per-node chain rule
// through the equilibrium, projection, BGK update and EDM force stays in FP32.
//
// Same mathematics as adjoint.cu (the FP32 CUDA-core adjoint):
//   lam_i(x - c_i) = [J_C(f(x))^T lam'(x)]_i,   dtheta += sum_x (dC/dtheta)^T lam'(x).
//
// A warpgroup owns a 128-node tile (thread r = node r = TMEM lane r) and runs
// five GEMMs with M = 128 nodes in four round trips:
//   1. x|1 . W1'^T (layer 1 recomputed) and dL/do . W3 = dL/dh2 (dL/do needs only
//      the incoming adjoint and rho), issued together;
//   2. h1|1 . W2'^T (layer 2), whose epilogue forms h2 = tanh and, with the
//      parked dL/dh2, dL/da2 = dL/dh2 (1 - h2^2);
//   3. dL/da2 . W2 -> *(1 - h1^2) = dL/da1;   4. dL/da1 . W1 = dL/dx.
// The network output o is not recomputed: the update f' = ... + (rho/tau) P o
// needs it only in the rho-derivative of its scaling, sum_i (dL/df'_i omega)
// (P o)_i = (dL/do . o) / rho with dL/do = rho omega P dL/df' (P symmetric),
// and dL/do . o = (W3^T dL/do) . h2 + dL/do . b3, where W3^T dL/do is the first
// backward GEMM's result: a dot product in the layer-2 epilogue, where dL/dh2
// meets h2, instead of a GEMM round trip.
// The weight gradients are three GEMMs with the NODES as the reduction
// dimension (K = 16 nodes per MMA), M = 64 hidden units, reading the same
// node-row operand buffers as MN-major matrices:
//   dW3^T += h2^T . dL/do,  [dW2 | db2] += dL/da2^T . [h1 | 1],  [dW1 | db1] += dL/da1^T . [x | 1]
// (db3 = sum dL/do on the CUDA cores).
//
// Organisation (one persistent CTA per SM): three warpgroups, each with one
// tile in flight and its own 128 tensor-memory columns (accumulator, dL/dh2
// then the layer-1 tanh derivative), plus three issuer warps, one per weight-gradient
// GEMM (dW3, dW2, dW1), each accumulating the whole CTA's sum of its matrix
// (112 columns in all).  A warpgroup signals the issuer concerned as soon as
// the operands of that GEMM are complete (dL/do, then dL/da2, then dL/da1) and
// carries on with its own chain; it waits for an issuer only before it
// overwrites a buffer that issuer's GEMM reads.  An issuer takes the
// warpgroups' GEMMs in a fixed order (tile, then warpgroup), so every sum is
// accumulated in the same order on every run; an issuer thread stalls until
// its GEMM has completed before it can poll again, which is why the three
// matrices have an issuer each.  dL/da1 reuses the h2 buffer once the dW3 GEMM
// has read it.
// Every wait is bounded: on a time-out all roles leave their loops, the
// tensor memory is freed and the timeout flag is set.
#include <cuda_bf16.h>

#include "kernels.h"
#include "lattice.cuh"
#include "umma.cuh"

namespace lbm {
namespace {

using namespace umma;

constexpr int WG_THREADS = 128;
constexpr int WGS = 3;                  // tile warpgroups per CTA
constexpr int DW_WARP = WGS * 4;        // warp index of the first weight-gradient issuer
constexpr int THREADS = WGS * WG_THREADS + 3 * 32;
constexpr int K1 = 16, K2 = 80;
constexpr uint32_t TMEM_COLS = 512;
// per-warpgroup block: GEMM accumulator (64 columns) and 64 columns that hold
// the first backward GEMM's result dL/dh2 until layer 1's epilogue, then the
// layer-1 tanh derivative 1 - h1^2 (bf16 pairs, 32 columns)
constexpr uint32_t C_D = 0, C_DH1 = 64, WG_COLS = 128;
// weight-gradient sums of the CTA (M = 64 accumulators)
constexpr uint32_t C_DW2 = WGS * WG_COLS, C_DW1 = C_DW2 + 80, C_DW3 = C_DW1 + 16;
static_assert(C_DW3 + 16 <= TMEM_COLS, "tensor memory layout");
constexpr uint32_t WAIT_LIMIT = 1u << 20;
enum { ST_DW3 = 0, ST_DW2 = 1, ST_DW1 = 2, STAGES = 3 };

struct __align__(16) WgBuffers {
  unsigned char a1[2][128 * K1 * 2];  // x | 1 | 0 (node rows), alternate tiles
  unsigned char h1[128 * K2 * 2];   // h1 | 1 | 0
  unsigned char h2[128 * 64 * 2];   // h2, then dL/da1
  unsigned char ob[128 * 16 * 2];   // dL/do | 0
  unsigned char a2b[128 * 64 * 2];  // dL/da2
};

struct __align__(1024) Smem {
  unsigned char w1[HIDDEN * K1 * 2];  // [64 x 16]  W1 | b1
  unsigned char w2[HIDDEN * K2 * 2];  // [64 x 80]  W2 | b2
  unsigned char w3t[HIDDEN * 16 * 2]; // [64 x 16]  [j][i] = W3[i][j]
  unsigned char w2t[HIDDEN * 64 * 2]; // [64 x 64]  [k][j] = W2[j][k]
  unsigned char w1t[16 * 64 * 2];     // [16 x 64]  [i][j] = W1[j][i]
  WgBuffers wb[WGS];
  unsigned long long bar[WGS];          // the warpgroup's own GEMMs (commit)
  unsigned long long rdy[WGS][STAGES];  // operands of a weight-gradient GEMM written
  unsigned long long dwd[WGS][STAGES];  // that GEMM has completed (commit)
  unsigned long long drain[STAGES];
  float db3[WGS * 4][9];
  float b3[16];                       // b3 rounded to bf16, as floats
  uint32_t taddr;
  int err;
};
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;
static_assert(SMEM_BYTES <= 227 * 1024, "adjoint shared memory too large");

__device__ __forceinline__ void store_bf16(unsigned char *base, int r, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + canon_offset(r, k, K)) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ void project9(float o[Q]) {
  float s = 0.f, sx = 0.f, sy = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    s += o[i];
    sx += (float)cx(i) * o[i];
    sy += (float)cy(i) * o[i];
  }
  const float k1 = -s * (1.0f / 9.0f), k2 = -sx * (1.0f / 6.0f), k3 = -sy * (1.0f / 6.0f);
#pragma unroll
  for (int i = 0; i < Q; ++i) o[i] += k1 + (float)cx(i) * k2 + (float)cy(i) * k3;
}

// Sums of a per-direction vector g against the partial derivatives of
// feq_i(rho, u) = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2).  feq_i is
// quadratic in c_i, so every such sum is a combination of the six weighted
// moments sum_i w_i g_i c_i^a c_i^b (monomials 1, c_x, c_y, c_x^2, c_x c_y,
// c_y^2): about 40 operations for the moments and 25 per velocity, instead of
// the 9 x 20 of a sum over directions.
struct GMom {
  float g0, gx, gy, gxx, gxy, gyy;
};
// Adds w_i g times the monomials of direction i (compile-time i).
__device__ __forceinline__ void gmom_add(GMom &s, int i, float g) {
  const float v = wf(i) * g;
  s.g0 += v;
  if (cx(i) != 0) {
    s.gx += cx(i) > 0 ? v : -v;
    s.gxx += v;
  }
  if (cy(i) != 0) {
    s.gy += cy(i) > 0 ? v : -v;
    s.gyy += v;
  }
  if (cx(i) * cy(i) != 0) s.gxy += cx(i) * cy(i) > 0 ? v : -v;
}
__device__ __forceinline__ GMom weighted_moments(const float g[Q]) {
  GMom s = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) gmom_add(s, i, g[i]);
  return s;
}
// sum_i g_i dfeq_i/drho, dfeq_i/du_x, dfeq_i/du_y at (rho, ux, uy)
__device__ __forceinline__ void feq_vjp(const GMom &s, float rho, float ux, float uy, float &sr,
                                        float &sx, float &sy) {
  const float usq = ux * ux + uy * uy;
  sr = s.g0 * (1.0f - 1.5f * usq) + 3.0f * (ux * s.gx + uy * s.gy) +
       4.5f * (ux * ux * s.gxx + 2.0f * ux * uy * s.gxy + uy * uy * s.gyy);
  sx = rho * (3.0f * s.gx + 9.0f * (ux * s.gxx + uy * s.gxy) - 3.0f * ux * s.g0);
  sy = rho * (3.0f * s.gy + 9.0f * (ux * s.gxy + uy * s.gyy) - 3.0f * uy * s.g0);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

#ifndef LBM_ADJ_TANH_EX2
#define LBM_ADJ_TANH_EX2 0
#endif
// tanh(a) and its derivative 1 - tanh(a)^2.
// Default: the hardware tanh.approx.f32 (one XU operation, 8 cycles per
// warp-instruction) and 1 - h^2 on the FMA pipe.  For a saturated unit the
// derivative then has an absolute error of ~1e-3 (h is good to ~2^-11
// relative), which is what matters for the chain rule: it scales the
// incoming gradient, so the error is ~1e-3 of that gradient, the size of the
// bf16 rounding of the backward operands.
// LBM_ADJ_TANH_EX2=1: t = e^{-2|a|}, r = 1/(1 + t), u = t r:
// tanh a = sign(a) (r - u), 1 - tanh^2 a = 4 u r (ex2 + rcp: 12 XU cycles per
// warp-instruction pair of values; keeps the derivative's relative accuracy).
__device__ __forceinline__ void tanh_and_slope(float a, float &h, float &dh) {
  if (LBM_ADJ_TANH_EX2) {
    float t, r;
    const float e = -2.8853900817779268f * fabsf(a);  // -2 log2(e) |a|
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(e));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + t));
    const float u = t * r;
    h = copysignf(r - u, a);
    dh = 4.0f * (u * r);
  } else {
    asm("tanh.approx.f32 %0, %1;" : "=f"(h) : "f"(a));
    dh = fmaf(-h, h, 1.0f);
  }
}

// Two units at once: h = tanh(a) per value, and 1 - h^2 for both in one
// packed fused multiply-add (the same rounding as two scalar ones).
__device__ __forceinline__ void tanh_and_slope2(float a0, float a1, float2 &h, float2 &dh) {
  if (LBM_ADJ_TANH_EX2) {
    tanh_and_slope(a0, h.x, dh.x);
    tanh_and_slope(a1, h.y, dh.y);
  } else {
    asm("tanh.approx.f32 %0, %1;" : "=f"(h.x) : "f"(a0));
    asm("tanh.approx.f32 %0, %1;" : "=f"(h.y) : "f"(a1));
    dh = __ffma2_rn(make_float2(-h.x, -h.y), h, make_float2(1.0f, 1.0f));
  }
}

// D (64 FP32 columns of this thread's row) -> h = tanh(D) in FP32 -> bf16 row of
// `dst` (K columns 0..63, the next GEMM's operand), and the derivative 1 - h^2,
// computed to a few ulp in FP32 and rounded to bf16 pairs, into 32 TMEM
// columns at tm_dh (the derivative of a saturated unit would lose its digits
// if it were formed from a rounded or approximate h).
__device__ __forceinline__ void tanh_row(uint32_t tm_row, unsigned char *dst, int r,
                                         uint32_t tm_dh) {
#pragma unroll
  for (int c = 0; c < HIDDEN; c += 32) {
    uint32_t v[32];
    tmem_ld32(tm_row + c, v);
    tmem_wait_ld();
    uint32_t p[16], q[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float2 h, dh;
      tanh_and_slope2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]), h, dh);
      p[e] = pack_bf16x2(h.x, h.y);
      q[e] = pack_bf16x2(dh.x, dh.y);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      *reinterpret_cast<uint4 *>(dst + canon_offset(r, c + 8 * e, K2)) =
          make_uint4(p[4 * e], p[4 * e + 1], p[4 * e + 2], p[4 * e + 3]);
    tmem_st16(tm_dh + c / 2, q);
  }
  tmem_wait_st();
}

// D (64 columns) * (1 - h^2), the derivative read back from tm_dh
// -> bf16 row of `dst` (row length 64).
__device__ __forceinline__ void dtanh_row(uint32_t tm_row, uint32_t tm_dh, unsigned char *dst,
                                          int r) {
#pragma unroll
  for (int c = 0; c < HIDDEN; c += 32) {
    uint32_t v[32], dh[16];
    tmem_ld32(tm_row + c, v);
    tmem_ld16(tm_dh + c / 2, dh);
    tmem_wait_ld();
    uint32_t p[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float2 g =
          __fmul2_rn(make_float2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1])),
                     make_float2(bf16_lo(dh[e]), bf16_hi(dh[e])));
      p[e] = pack_bf16x2(g.x, g.y);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      *reinterpret_cast<uint4 *>(dst + canon_offset(r, c + 8 * e, 64)) =
          make_uint4(p[4 * e], p[4 * e + 1], p[4 * e + 2], p[4 * e + 3]);
  }
}

// The first backward GEMM's result dL/dh2 (64 accumulator columns at tm)
// -> bf16 row r of `g` (row length 64), where the layer-2 epilogue reads it.
__device__ __forceinline__ void park_row(uint32_t tm, unsigned char *g, int r) {
#pragma unroll
  for (int c = 0; c < HIDDEN; c += 32) {
    uint32_t v[32];
    tmem_ld32(tm + c, v);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 4; ++e)
      *reinterpret_cast<uint4 *>(g + canon_offset(r, c + 8 * e, 64)) =
          make_uint4(pack_bf16x2(__uint_as_float(v[8 * e]), __uint_as_float(v[8 * e + 1])),
                     pack_bf16x2(__uint_as_float(v[8 * e + 2]), __uint_as_float(v[8 * e + 3])),
                     pack_bf16x2(__uint_as_float(v[8 * e + 4]), __uint_as_float(v[8 * e + 5])),
                     pack_bf16x2(__uint_as_float(v[8 * e + 6]), __uint_as_float(v[8 * e + 7])));
  }
}

// Layer-2 epilogue with the reverse step fused: h2 = tanh(D) as the bf16 row
// r of `hdst` (row length 64, the dW3 operand), and with g = dL/dh2 from the bf16 row r of
// `g`, dL/da2 = g (1 - h2^2) written back over g.  Returns sum_k g_k h2_k
// (h2 as stored), the output's term of the rho-derivative before its 1/rho.
__device__ __forceinline__ float tanh_grad_row(uint32_t tm_row, unsigned char *hdst,
                                               unsigned char *g, int r) {
  float2 dot = make_float2(0.f, 0.f);  // even and odd units
#pragma unroll
  for (int c = 0; c < HIDDEN; c += 32) {
    uint32_t v[32];
    tmem_ld32(tm_row + c, v);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint4 gv = *reinterpret_cast<const uint4 *>(g + canon_offset(r, c + 8 * e, 64));
      const uint32_t gw[4] = {gv.x, gv.y, gv.z, gv.w};
      uint32_t hp[4], ap[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 h, dh;
        tanh_and_slope2(__uint_as_float(v[8 * e + 2 * q]), __uint_as_float(v[8 * e + 2 * q + 1]), h,
                        dh);
        hp[q] = pack_bf16x2(h.x, h.y);
        const float2 g = make_float2(bf16_lo(gw[q]), bf16_hi(gw[q]));
        const float2 a = __fmul2_rn(g, dh);
        ap[q] = pack_bf16x2(a.x, a.y);
        dot = __ffma2_rn(g, make_float2(bf16_lo(hp[q]), bf16_hi(hp[q])), dot);
      }
      *reinterpret_cast<uint4 *>(hdst + canon_offset(r, c + 8 * e, 64)) =
          make_uint4(hp[0], hp[1], hp[2], hp[3]);
      *reinterpret_cast<uint4 *>(g + canon_offset(r, c + 8 * e, 64)) =
          make_uint4(ap[0], ap[1], ap[2], ap[3]);
    }
  }
  return dot.x + dot.y;
}

struct TilePos {
  int b, y, x0;
  __device__ __forceinline__ void advance(int nx, int ny) {
    x0 += WG_THREADS;
    if (x0 >= nx) {
      x0 = 0;
      if (++y == ny) {
        y = 0;
        ++b;
      }
    }
  }
};

__device__ __forceinline__ void prefetch_l2(const float *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait of one thread; gives up early once another role has recorded
// an error, and records one itself on a time-out.
__device__ __forceinline__ bool wait_flag(uint32_t bar, uint32_t parity, volatile int *err) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 15u && *err) return false;
  }
  atomicOr(const_cast<int *>(err), 1);
  return false;
}
// Warpgroup-wide wait on one or two barriers: the leader polls, the named
// barrier hands every thread the same verdict.
__device__ __forceinline__ bool wg_wait(uint32_t b0, uint32_t p0, uint32_t b1, uint32_t p1,
                                        bool two, bool leader, uint32_t bar_id,
                                        volatile int *err) {
  bool fail = false;
  if (leader) {
    fail = !wait_flag(b0, p0, err);
    if (!fail && two) fail = !wait_flag(b1, p1, err);
  }
  const bool any = barrier_any(bar_id, WG_THREADS, fail);
  fence_after_sync();
  return !any;
}

__global__ void __launch_bounds__(THREADS, 1)
    k_adjoint_tc(const float *__restrict__ state, const float *__restrict__ lam_next,
                 float *__restrict__ lam_out, int nx, int ny, int batch, CollideParams p,
                 MlpF32 w, float *__restrict__ partials, int accumulate, int *timeout_flag) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *err = &S.err;

  // ---- prologue: weights in the five operand layouts, and b3
  for (int e = tid; e < HIDDEN * K1; e += THREADS) {
    const int n = e / K1, k = e % K1;
    store_bf16(S.w1, n, k, K1, k < 9 ? w.w1[n * 9 + k] : (k == 9 ? w.b1[n] : 0.f));
  }
  for (int e = tid; e < HIDDEN * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    store_bf16(S.w2, n, k, K2, k < HIDDEN ? w.w2[n * HIDDEN + k] : (k == HIDDEN ? w.b2[n] : 0.f));
  }
  if (tid < 16) S.b3[tid] = tid < 9 ? __bfloat162float(__float2bfloat16_rn(w.b3[tid])) : 0.f;
  for (int e = tid; e < HIDDEN * 16; e += THREADS) {
    const int j = e / 16, i = e % 16;
    store_bf16(S.w3t, j, i, 16, i < 9 ? w.w3[i * HIDDEN + j] : 0.f);
  }
  for (int e = tid; e < HIDDEN * HIDDEN; e += THREADS) {
    const int k = e / HIDDEN, j = e % HIDDEN;
    store_bf16(S.w2t, k, j, 64, w.w2[j * HIDDEN + k]);
  }
  for (int e = tid; e < 16 * HIDDEN; e += THREADS) {
    const int i = e / HIDDEN, j = e % HIDDEN;
    store_bf16(S.w1t, i, j, 64, i < 9 ? w.w1[j * 9 + i] : 0.f);
  }
  if (warp < DW_WARP) {
    // constant columns 64..79 of the h1 rows: 1, 0, ..., 0
    WgBuffers &B = S.wb[warp >> 2];
    const int r = tid & 127;
    *reinterpret_cast<uint4 *>(B.h1 + canon_offset(r, 64, K2)) = make_uint4(0x3F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(B.h1 + canon_offset(r, 72, K2)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int g = 0; g < WGS; ++g) {
      mbar_init(smem_u32(&S.bar[g]), 1);
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(smem_u32(&S.rdy[g][s]), 1);
        mbar_init(smem_u32(&S.dwd[g][s]), 1);
      }
    }
    for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&S.drain[s]), 1);
    S.err = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&S.taddr), TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = S.taddr;
  // The prologue above reads only the weights.  Launched as a programmatic
  // dependent of the previous kernel of the backward pass, this CTA waits for
  // it here, before its first access to the states, adjoints, partial sums or
  // flags, and lets the next launch start its own prologue as SMs free up.
  griddep_wait();
  griddep_launch_dependents();

  const int plane = nx * ny;
  const int tiles_x = (nx + WG_THREADS - 1) / WG_THREADS;
  const int ntiles = tiles_x * ny * batch;
  const int nwg = gridDim.x * WGS;
  auto range = [&](int g, int &begin, int &count) {
    const int gwg = blockIdx.x * WGS + g;
    const int per = ntiles / nwg, extra = ntiles % nwg;
    begin = gwg * per + min(gwg, extra);
    count = per + (gwg < extra ? 1 : 0);
  };
  // weight-gradient GEMMs: M = 64, both operands MN-major (bits 15, 16)
  constexpr uint32_t IDW80 = idesc_bf16_f32(64, 80) | (1u << 15) | (1u << 16);
  constexpr uint32_t IDW16 = idesc_bf16_f32(64, 16) | (1u << 15) | (1u << 16);
  float db3[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) db3[i] = 0.f;
  bool any_tiles = false;

  if (warp >= DW_WARP) {
    // ---------------- weight-gradient issuers: warp DW_WARP + s runs stage s
    const int s = warp - DW_WARP;
    if (lane == 0) {
      int cnt[WGS];
      int rounds = 0;
#pragma unroll
      for (int g = 0; g < WGS; ++g) {
        int b;
        range(g, b, cnt[g]);
        rounds = max(rounds, cnt[g]);
      }
      uint32_t par = 0;  // bit g: parity of rdy[g][s]
      bool started = false, ok = true;
      const uint32_t acc_col = s == ST_DW3 ? C_DW3 : (s == ST_DW2 ? C_DW2 : C_DW1);
      const uint32_t id = s == ST_DW2 ? IDW80 : IDW16;
      for (int k = 0; k < rounds && ok; ++k) {
#pragma unroll
        for (int g = 0; g < WGS; ++g) {
          if (!ok || k >= cnt[g]) continue;
          if (!wait_flag(smem_u32(&S.rdy[g][s]), (par >> g) & 1u, err)) {
            ok = false;
            continue;
          }
          par ^= 1u << g;
          fence_after_sync();
          const WgBuffers &B = S.wb[g];
          // operands: dW3^T = h2^T dL/do; dW2 = dL/da2^T [h1|1]; dW1 = dL/da1^T [x|1]
          // (dL/da1 lives in the h2 buffer)
          uint32_t sa, sb, a_lbo, b_lbo;
          if (s == ST_DW3) {
            sa = smem_u32(B.h2), a_lbo = 1024, sb = smem_u32(B.ob), b_lbo = 256;
          } else if (s == ST_DW2) {
            sa = smem_u32(B.a2b), a_lbo = 1024, sb = smem_u32(B.h1), b_lbo = 1280;
          } else {
            sa = smem_u32(B.h2), a_lbo = 1024, sb = smem_u32(B.a1[k & 1]), b_lbo = 256;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q)
            mma_bf16(tmem + acc_col, smem_desc(sa + 2 * a_lbo * q, a_lbo, 128),
                     smem_desc(sb + 2 * b_lbo * q, b_lbo, 128), id, (started || q > 0) ? 1u : 0u);
          mma_commit(smem_u32(&S.dwd[g][s]));
          started = true;
        }
      }
      if (started) {  // every weight-gradient MMA done before the sums are read
        mma_commit(smem_u32(&S.drain[s]));
        if (!mbar_wait_bounded(smem_u32(&S.drain[s]), 0, WAIT_LIMIT))
          atomicOr(const_cast<int *>(err), 1);
      }
    }
    __syncwarp();
  } else {
    // ---------------- tile warpgroups
    const int wg = warp >> 2;
    const int r = tid & 127;
#ifndef LBM_ADJ_LEADER_SPREAD
#define LBM_ADJ_LEADER_SPREAD 1
#endif
    // the thread that issues and waits for the warpgroup's GEMMs
    const bool leader = LBM_ADJ_LEADER_SPREAD ? r == 32 * ((wg + 1) & 3) : r == 0;
    const uint32_t bar_id = 1 + wg;
    WgBuffers &B = S.wb[wg];
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t tm_wg = tmem + (uint32_t)(wg * WG_COLS);
    const uint32_t tm_row = tm_wg + C_D + lane_off;
    const uint32_t bar = smem_u32(&S.bar[wg]);
    const uint32_t s_h1 = smem_u32(B.h1), s_h2 = smem_u32(B.h2);
    const uint32_t s_ob = smem_u32(B.ob), s_a2b = smem_u32(B.a2b);
    const uint32_t s_w1 = smem_u32(S.w1), s_w2 = smem_u32(S.w2);
    const uint32_t s_w3t = smem_u32(S.w3t), s_w2t = smem_u32(S.w2t), s_w1t = smem_u32(S.w1t);
    constexpr uint32_t ID64 = idesc_bf16_f32(128, 64), ID16 = idesc_bf16_f32(128, 16);
    unsigned char *a1b = B.h2;  // dL/da1 takes the h2 buffer once dW3 has read it
    int t_begin, count;
    range(wg, t_begin, count);
    any_tiles = count > 0;
    TilePos T;
    T.x0 = (t_begin % tiles_x) * WG_THREADS;
    T.y = (t_begin / tiles_x) % ny;
    T.b = t_begin / (tiles_x * ny);
    const float omega = p.omega;
    uint32_t phase = 0, dpar = 0;  // own GEMMs; bit s: parity of dwd[wg][s]
    bool pending = false;          // the leader has an own commit outstanding

// the warpgroup's own GEMM: wait for its commit
#define WAIT_OWN_OR_BREAK()                                                    \
  if (!wg_wait(bar, phase, 0, 0, false, leader, bar_id, err)) break;            \
  phase ^= 1;                                                                   \
  pending = false;
// all operand rows written: make them visible to the tensor core
#define OPERANDS_READY()   \
  fence_proxy_async();     \
  fence_before_sync();     \
  named_barrier(bar_id, WG_THREADS);

    float dn[Q], pbn[Q];  // the next tile's inputs
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      dn[i] = 0.f;
      pbn[i] = 0.f;
    }
    for (int it = 0; it < count; ++it) {
      // The previous tile's weight-gradient GEMMs may still be reading its
      // buffers: dW2 reads h1 and dL/da2 (waited for before this tile's
      // layer-1 epilogue writes them), dW1 reads its x and dL/da1 (x
      // alternates between two buffers; dL/da1 shares the h2 buffer, waited
      // for before the layer-2 epilogue).  dW3 was waited for within that tile.
      unsigned char *a1 = B.a1[it & 1];
      const uint32_t s_a1 = smem_u32(a1);
      const int x = T.x0 + r;
      const bool active = x < nx;
      const int ym = T.y == 0 ? ny - 1 : T.y - 1, yp = T.y == ny - 1 ? 0 : T.y + 1;
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x >= nx - 1 ? 0 : x + 1;
      // this tile's populations and incoming adjoint: loaded during the
      // previous tile's last GEMM, or here for the first tile
      float d[Q], pb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        d[i] = dn[i];
        pb[i] = pbn[i];
      }
      if (active && it == 0) {
        const float *gb = state + (size_t)T.b * Q * plane;
        const float *lb = lam_next + (size_t)T.b * Q * plane + T.y * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
          const int ys = cy(i) == 0 ? T.y : (cy(i) == 1 ? ym : yp);
          d[i] = __ldg(gb + (size_t)i * plane + ys * nx + xs);
          pb[i] = __ldg(lb + (size_t)i * plane);
        }
      }
      // ---- the next tile's inputs are prefetched into the L2 cache now, so
      // that its loads return from L2 (no registers are held for them)
      if (it + 1 < count) {
        TilePos N = T;
        N.advance(nx, ny);
        const int xn = N.x0 + r;
        if (xn < nx) {
          const int nym = N.y == 0 ? ny - 1 : N.y - 1, nyp = N.y == ny - 1 ? 0 : N.y + 1;
          const int nxm = xn == 0 ? nx - 1 : xn - 1, nxp = xn >= nx - 1 ? 0 : xn + 1;
          const float *gb = state + (size_t)N.b * Q * plane;
          const float *lb = lam_next + (size_t)N.b * Q * plane + N.y * nx + xn;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int xs = cx(i) == 0 ? xn : (cx(i) == 1 ? nxm : nxp);
            const int ys = cy(i) == 0 ? N.y : (cy(i) == 1 ? nym : nyp);
            prefetch_l2(gb + (size_t)i * plane + ys * nx + xs);
            prefetch_l2(lb + (size_t)i * plane);
          }
        }
      }
      // ---- forward recompute: moments, equilibrium, layer-1 operand
      Moments m;
      float inv_rho;
      {
        const float drho =
            ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        m.drho = drho;
        m.rho = 1.0f + drho;
        inv_rho = 1.0f / m.rho;
        m.ux = jx * inv_rho;
        m.uy = jy * inv_rho;
        float deq[Q], xin[Q];
        shifted_feq(m, deq);
#pragma unroll
        for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * inv_rho;
        *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 0, K1)) =
            make_uint4(pack_bf16x2(xin[0], xin[1]), pack_bf16x2(xin[2], xin[3]),
                       pack_bf16x2(xin[4], xin[5]), pack_bf16x2(xin[6], xin[7]));
        *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 8, K1)) =
            make_uint4(pack_bf16x2(xin[8], 1.0f), 0u, 0u, 0u);
      }
      // ---- dL/do (FP32) needs only the incoming adjoint and rho, so its GEMM
      // (dL/dh2 = dL/do . W3) runs beside layer 1
      // post = d + omega (deq - d) + rho omega ohat + fext(rho, u)
      float rhob = 0.f, uxb = 0.f, uyb = 0.f, ob_b3 = 0.f;
      {
        float ob[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) ob[i] = m.rho * omega * pb[i];
        if (p.force) {
          // f_ext = feq(rho, u + a) - feq(rho, u), a = (fx/rho, 0): the
          // differences of the two sums, written without cancellation
          // (s = 2 u_x + a_x), and the rho-dependence of a
          const float fx = __ldg(p.force + T.y);
          const float ax = fx * inv_rho;
          const float sxs = 2.0f * m.ux + ax, uxs = m.ux + ax;
          const GMom q = weighted_moments(pb);
          const float sx1 =
              m.rho * (3.0f * q.gx + 9.0f * (uxs * q.gxx + m.uy * q.gxy) - 3.0f * uxs * q.g0);
          rhob += ax * (3.0f * q.gx + 4.5f * (sxs * q.gxx + 2.0f * m.uy * q.gxy) -
                        1.5f * sxs * q.g0) -
                  ax * inv_rho * sx1;
          uxb += m.rho * ax * (9.0f * q.gxx - 3.0f * q.g0);
          uyb += m.rho * ax * 9.0f * q.gxy;
        }
        project9(ob);  // dL/do = P dL/dohat (P symmetric)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          db3[i] += ob[i];
          ob_b3 = fmaf(ob[i], S.b3[i], ob_b3);
        }
        *reinterpret_cast<uint4 *>(B.ob + canon_offset(r, 0, 16)) =
            make_uint4(pack_bf16x2(ob[0], ob[1]), pack_bf16x2(ob[2], ob[3]),
                       pack_bf16x2(ob[4], ob[5]), pack_bf16x2(ob[6], ob[7]));
        *reinterpret_cast<uint4 *>(B.ob + canon_offset(r, 8, 16)) =
            make_uint4(pack_bf16x2(ob[8], 0.0f), 0u, 0u, 0u);
      }
      OPERANDS_READY()
      if (leader) {
        fence_after_sync();
        mma_bf16(tm_wg + C_D, smem_desc(s_a1, 128, 16 * K1), smem_desc(s_w1, 128, 16 * K1), ID64,
                 0);
        // into the derivative columns, free until layer 1's epilogue
        mma_bf16(tm_wg + C_DH1, smem_desc(s_ob, 128, 256), smem_desc(s_w3t, 128, 256), ID64, 0);
        mma_commit(bar);
        pending = true;
      }
      // own GEMMs, and the previous tile's dW2 (it reads h1 and dL/da2)
      if (!wg_wait(bar, phase, smem_u32(&S.dwd[wg][ST_DW2]), (dpar >> ST_DW2) & 1u, it > 0, leader,
                   bar_id, err))
        break;
      phase ^= 1;
      pending = false;
      if (it > 0) dpar ^= 1u << ST_DW2;
      park_row(tm_wg + C_DH1 + lane_off, B.a2b, r);  // read before the derivative overwrites it
      tanh_row(tm_row, B.h1, r, tm_wg + C_DH1 + lane_off);
      OPERANDS_READY()
      if (leader) {
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < K2 / 16; ++s)
          mma_bf16(tm_wg + C_D, smem_desc(s_h1 + 256 * s, 128, 16 * K2),
                   smem_desc(s_w2 + 256 * s, 128, 16 * K2), ID64, s > 0);
        mma_commit(bar);
        pending = true;
      }
      // own GEMM, and the previous tile's dW1 (it reads dL/da1 in the h2 buffer)
      if (!wg_wait(bar, phase, smem_u32(&S.dwd[wg][ST_DW1]), (dpar >> ST_DW1) & 1u, it > 0, leader,
                   bar_id, err))
        break;
      phase ^= 1;
      pending = false;
      if (it > 0) dpar ^= 1u << ST_DW1;
      rhob = fmaf(tanh_grad_row(tm_row, B.h2, B.a2b, r) + ob_b3, inv_rho, rhob);
      OPERANDS_READY()
      if (leader) {
        mbar_arrive(smem_u32(&S.rdy[wg][ST_DW3]));  // h2 and dL/do complete
        mbar_arrive(smem_u32(&S.rdy[wg][ST_DW2]));  // dL/da2 and h1 complete
        fence_after_sync();
        // dL/da1 (before the tanh derivative) = dL/da2 . W2
#pragma unroll
        for (int s = 0; s < 4; ++s)
          mma_bf16(tm_wg + C_D, smem_desc(s_a2b + 256 * s, 128, 1024),
                   smem_desc(s_w2t + 256 * s, 128, 1024), ID64, s > 0);
        mma_commit(bar);
        pending = true;
      }
      // own GEMM, and dW3 (it reads h2, which dL/da1 overwrites next)
      if (!wg_wait(bar, phase, smem_u32(&S.dwd[wg][ST_DW3]), (dpar >> ST_DW3) & 1u, true, leader,
                   bar_id, err))
        break;
      phase ^= 1;
      pending = false;
      dpar ^= 1u << ST_DW3;
      dtanh_row(tm_row, tm_wg + C_DH1 + lane_off, a1b, r);
      OPERANDS_READY()
      if (leader) {
        mbar_arrive(smem_u32(&S.rdy[wg][ST_DW1]));  // dL/da1 and x complete
        fence_after_sync();
        // dL/dx = dL/da1 . W1
#pragma unroll
        for (int s = 0; s < 4; ++s)
          mma_bf16(tm_wg + C_D, smem_desc(s_h2 + 256 * s, 128, 1024),
                   smem_desc(s_w1t + 256 * s, 128, 1024), ID16, s > 0);
        mma_commit(bar);
        pending = true;
      }
      // ---- the next tile's inputs into registers while the last GEMM runs
      // (they were prefetched into the L2 cache at this tile's start)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        dn[i] = 0.f;
        pbn[i] = 0.f;
      }
      if (it + 1 < count) {
        TilePos N = T;
        N.advance(nx, ny);
        const int xn = N.x0 + r;
        if (xn < nx) {
          const int nym = N.y == 0 ? ny - 1 : N.y - 1, nyp = N.y == ny - 1 ? 0 : N.y + 1;
          const int nxm = xn == 0 ? nx - 1 : xn - 1, nxp = xn >= nx - 1 ? 0 : xn + 1;
          const float *gb = state + (size_t)N.b * Q * plane;
          const float *lb = lam_next + (size_t)N.b * Q * plane + N.y * nx + xn;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const int xs = cx(i) == 0 ? xn : (cx(i) == 1 ? nxm : nxp);
            const int ys = cy(i) == 0 ? N.y : (cy(i) == 1 ? nym : nyp);
            dn[i] = __ldg(gb + (size_t)i * plane + ys * nx + xs);
            pbn[i] = __ldg(lb + (size_t)i * plane);
          }
        }
      }
      WAIT_OWN_OR_BREAK()
      // ---- dL/dx -> rest of the chain rule (FP32), scatter lam to x - c_i
      {
        uint32_t xv[16];
        tmem_ld16(tm_row, xv);
        tmem_wait_ld();
        float deq[Q];
        shifted_feq(m, deq);
        float fb[Q];
        GMom q = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // moments of dL/dfeq
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float xb = __uint_as_float(xv[i]) * inv_rho;
          const float xin = (d[i] - deq[i]) * inv_rho;
          fb[i] = pb[i] * (1.0f - omega) + xb;
          gmom_add(q, i, pb[i] * omega - xb);
          rhob -= xb * xin;
        }
        {
          float sr, sx, sy;
          feq_vjp(q, m.rho, m.ux, m.uy, sr, sx, sy);
          rhob += sr;
          uxb += sx;
          uyb += sy;
        }
        const float jxb = uxb * inv_rho, jyb = uyb * inv_rho;
        rhob -= (uxb * m.ux + uyb * m.uy) * inv_rho;
        if (active) {
          float *lo = lam_out + (size_t)T.b * Q * plane;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const float v = fb[i] + rhob + (float)cx(i) * jxb + (float)cy(i) * jyb;
            const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
            const int ys = cy(i) == 0 ? T.y : (cy(i) == 1 ? ym : yp);
            lo[(size_t)i * plane + ys * nx + xs] = v;  // lam_i(x - c_i)
          }
        }
      }
      T.advance(nx, ny);
    }
#undef WAIT_OWN_OR_BREAK
#undef OPERANDS_READY
    // after a time-out: let this warpgroup's own MMAs finish before the
    // tensor memory is freed
    if (leader && pending) mbar_wait_bounded(bar, phase, WAIT_LIMIT);
  }

  // ---- db3: per-warp sums of dL/do
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float v = db3[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0 && warp < DW_WARP) S.db3[warp][i] = v;
  }
  // ---- teardown: every role has left its loop, the issuer has drained
  fence_before_sync();
  const int any = __syncthreads_or(any_tiles ? 1 : 0);
  fence_after_sync();
  const bool have = any && !S.err;
  float *row = partials + (size_t)blockIdx.x * NPARAMS;
  if (warp < 4) {
    // M = 64 accumulators: row j lives in lane 32 (j / 16) + j % 16
    const uint32_t lo = (uint32_t)(32 * warp) << 16;
    const int j = 16 * warp + lane;
#pragma unroll 1
    for (int c = 0; c < 7; ++c) {
      uint32_t v[16];
      const uint32_t col = c < 5 ? C_DW2 + 16 * c : (c == 5 ? C_DW1 : C_DW3);
      tmem_ld16(tmem + col + lo, v);
      tmem_wait_ld();
      if (lane < 16) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float g = have ? __uint_as_float(v[k]) : 0.f;
          float *dst = nullptr;
          if (c < 4) {
            dst = row + OFF_W2 + j * HIDDEN + 16 * c + k;
          } else if (c == 4) {
            if (k == 0) dst = row + OFF_B2 + j;
          } else if (c == 5) {
            if (k < 9) dst = row + OFF_W1 + j * 9 + k;
            else if (k == 9) dst = row + OFF_B1 + j;
          } else {
            if (k < 9) dst = row + OFF_W3 + k * HIDDEN + j;
          }
          if (dst) *dst = accumulate ? *dst + g : g;
        }
      }
    }
  }
  if (tid < 9) {
    float g = 0.f;
    for (int k = 0; k < WGS * 4; ++k) g += S.db3[k][tid];
    if (!have) g = 0.f;
    row[OFF_B3 + tid] = accumulate ? row[OFF_B3 + tid] + g : g;
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
  if (tid == 0 && S.err) atomicOr(timeout_flag, 1);
}

}  // namespace

int adjoint_tc_rows(const Grid &g, int sms) {
  const long long tiles = (long long)((g.nx + WG_THREADS - 1) / WG_THREADS) * g.ny * g.batch;
  long long ctas = (tiles + WGS - 1) / WGS;
  if (ctas > sms) ctas = sms;
  return (int)ctas;  // one row of partial sums per CTA
}

cudaError_t launch_adjoint_tc(const Grid &g, const float *state_n, const float *lam_next,
                              float *lam_out, const CollideParams &p, const MlpF32 &w,
                              float *dw_partials, int rows, int accumulate, int *timeout_flag,
                              cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if ((long long)g.nx * g.ny * g.batch * Q >= (1LL << 31)) return cudaErrorInvalidValue;
  // a programmatic dependent of the previous kernel on the stream: in the
  // backward pass that is always one of this library's (the push, a recompute
  // step or the previous adjoint step), none of which writes the weights that
  // the prologue reads before its wait
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)rows);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_adjoint_tc, state_n, lam_next, lam_out, g.nx, g.ny, g.batch, p,
                            w, dw_partials, accumulate, timeout_flag);
}

}  // namespace lbm
