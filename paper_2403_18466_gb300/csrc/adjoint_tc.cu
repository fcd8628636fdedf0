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
// nine GEMMs with M = 128 nodes:
//   forward recompute   x|1 . W1'^T -> tanh -> h1|1 . W2'^T -> tanh -> h2|1 . W3'^T = o
//   backward            dL/do . W3 -> *(1-h2^2) = dL/da2 ;  dL/da2 . W2 -> *(1-h1^2) = dL/da1 ;
//                       dL/da1 . W1 = dL/dx
// and then three weight-gradient GEMMs with the NODES as the reduction
// dimension (K = 128), M = 64 hidden units, reading the same node-row operand
// buffers as MN-major matrices, accumulated in tensor memory over all of the
// warpgroup's tiles:
//   [dW2 | db2] += dL/da2^T . [h1 | 1],  [dW1 | db1] += dL/da1^T . [x | 1],
//   dW3^T += h2^T . dL/do                 (db3 = sum dL/do on the CUDA cores)
// Each warpgroup finally adds its sums to its own row of partial sums, which a
// fixed-order reduction turns into dtheta (bitwise reproducible).
#include <cuda_bf16.h>

#include "kernels.h"
#include "lattice.cuh"
#include "umma.cuh"

namespace lbm {
namespace {

using namespace umma;

constexpr int WG_THREADS = 128;
constexpr int WGS = 2;
constexpr int THREADS = WGS * WG_THREADS;
constexpr int K1 = 16, K2 = 80;
constexpr uint32_t TMEM_COLS = 512;  // 256 per warpgroup
// per-warpgroup column offsets: GEMM accumulator, the weight-gradient sums,
// and the tanh derivatives 1 - h^2 of both hidden layers (bf16 pairs)
constexpr uint32_t C_D = 0, C_DW2 = 64, C_DW1 = 144, C_DW3 = 160, C_DH1 = 176, C_DH2 = 208;
constexpr uint32_t WAIT_LIMIT = 1u << 20;

struct __align__(16) WgBuffers {
  unsigned char a1[128 * K1 * 2];   // x | 1 | 0        (node rows)
  unsigned char h1[128 * K2 * 2];   // h1 | 1 | 0
  unsigned char h2[128 * K2 * 2];   // h2 | 1 | 0
  unsigned char ob[128 * 16 * 2];   // dL/do | 0
  unsigned char a2b[128 * 64 * 2];  // dL/da2
  unsigned char a1b[128 * 64 * 2];  // dL/da1
};

struct __align__(1024) Smem {
  unsigned char w1[HIDDEN * K1 * 2];  // [64 x 16]  W1 | b1
  unsigned char w2[HIDDEN * K2 * 2];  // [64 x 80]  W2 | b2
  unsigned char w3[16 * K2 * 2];      // [16 x 80]  W3 | b3
  unsigned char w3t[HIDDEN * 16 * 2]; // [64 x 16]  [j][i] = W3[i][j]
  unsigned char w2t[HIDDEN * 64 * 2]; // [64 x 64]  [k][j] = W2[j][k]
  unsigned char w1t[16 * 64 * 2];     // [16 x 64]  [i][j] = W1[j][i]
  WgBuffers wb[WGS];
  unsigned long long bar[WGS];
  float db3[WGS][4][9];
  uint32_t taddr;
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

// Partial derivatives of feq_i(rho, u) = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2).
__device__ __forceinline__ void feq_partials(float rho, float ux, float uy, int i, float &dr,
                                             float &dux, float &duy) {
  const float cu = (float)cx(i) * ux + (float)cy(i) * uy;
  const float usq = ux * ux + uy * uy;
  dr = wf(i) * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * usq);
  dux = wf(i) * rho * (3.0f * (float)cx(i) + 9.0f * cu * (float)cx(i) - 3.0f * ux);
  duy = wf(i) * rho * (3.0f * (float)cy(i) + 9.0f * cu * (float)cy(i) - 3.0f * uy);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

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
      float h0, h1, d0, d1;
      tanh_and_derivative(__uint_as_float(v[2 * e]), h0, d0);
      tanh_and_derivative(__uint_as_float(v[2 * e + 1]), h1, d1);
      p[e] = pack_bf16x2_alu(h0, h1);
      q[e] = pack_bf16x2_alu(d0, d1);
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
    for (int e = 0; e < 16; ++e)
      p[e] = pack_bf16x2(__uint_as_float(v[2 * e]) * bf16_lo(dh[e]),
                         __uint_as_float(v[2 * e + 1]) * bf16_hi(dh[e]));
#pragma unroll
    for (int e = 0; e < 4; ++e)
      *reinterpret_cast<uint4 *>(dst + canon_offset(r, c + 8 * e, 64)) =
          make_uint4(p[4 * e], p[4 * e + 1], p[4 * e + 2], p[4 * e + 3]);
  }
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

__global__ void __launch_bounds__(THREADS, 1)
    k_adjoint_tc(const float *__restrict__ state, const float *__restrict__ lam_next,
                 float *__restrict__ lam_out, int nx, int ny, int batch, CollideParams p,
                 MlpF32 w, float *__restrict__ partials, int accumulate, int *timeout_flag) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int wg = tid / WG_THREADS;
  const int r = tid % WG_THREADS;
  const int warp_in_wg = r / 32;

  // ---- prologue: weights in the six operand layouts
  for (int e = tid; e < HIDDEN * K1; e += THREADS) {
    const int n = e / K1, k = e % K1;
    store_bf16(S.w1, n, k, K1, k < 9 ? w.w1[n * 9 + k] : (k == 9 ? w.b1[n] : 0.f));
  }
  for (int e = tid; e < HIDDEN * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    store_bf16(S.w2, n, k, K2, k < HIDDEN ? w.w2[n * HIDDEN + k] : (k == HIDDEN ? w.b2[n] : 0.f));
  }
  for (int e = tid; e < 16 * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    float v = 0.f;
    if (n < 9) v = k < HIDDEN ? w.w3[n * HIDDEN + k] : (k == HIDDEN ? w.b3[n] : 0.f);
    store_bf16(S.w3, n, k, K2, v);
  }
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
  WgBuffers &B = S.wb[wg];
  // constant columns 64..79 of the h1 / h2 rows: 1, 0, ..., 0
  for (unsigned char *hb : {B.h1, B.h2}) {
    *reinterpret_cast<uint4 *>(hb + canon_offset(r, 64, K2)) = make_uint4(0x3F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(hb + canon_offset(r, 72, K2)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int k = 0; k < WGS; ++k) mbar_init(smem_u32(&S.bar[k]), 1);
    fence_mbarrier_init();
  }
  if (tid < 32) {
    tmem_alloc(smem_u32(&S.taddr), TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();

  const uint32_t tm_wg = S.taddr + (uint32_t)(wg * 256);
  const uint32_t lane_off = (uint32_t)(32 * warp_in_wg) << 16;
  const uint32_t tm_row = tm_wg + C_D + lane_off;
  const uint32_t bar = smem_u32(&S.bar[wg]);
  const uint32_t bar_id = 1 + wg;
  const bool leader = r == 0;
  const uint32_t s_a1 = smem_u32(B.a1), s_h1 = smem_u32(B.h1), s_h2 = smem_u32(B.h2);
  const uint32_t s_ob = smem_u32(B.ob), s_a2b = smem_u32(B.a2b), s_a1b = smem_u32(B.a1b);
  const uint32_t s_w1 = smem_u32(S.w1), s_w2 = smem_u32(S.w2), s_w3 = smem_u32(S.w3);
  const uint32_t s_w3t = smem_u32(S.w3t), s_w2t = smem_u32(S.w2t), s_w1t = smem_u32(S.w1t);
  constexpr uint32_t ID64 = idesc_bf16_f32(128, 64), ID16 = idesc_bf16_f32(128, 16);
  // weight-gradient GEMMs: M = 64, both operands MN-major (bits 15, 16)
  constexpr uint32_t IDW80 = idesc_bf16_f32(64, 80) | (1u << 15) | (1u << 16);
  constexpr uint32_t IDW16 = idesc_bf16_f32(64, 16) | (1u << 15) | (1u << 16);

  const int plane = nx * ny;
  const int tiles_x = (nx + WG_THREADS - 1) / WG_THREADS;
  const int ntiles = tiles_x * ny * batch;
  const int nwg = gridDim.x * WGS;
  const int gwg = blockIdx.x * WGS + wg;
  const int per = ntiles / nwg, extra = ntiles % nwg;
  const int t_begin = gwg * per + min(gwg, extra);
  const int count = per + (gwg < extra ? 1 : 0);
  TilePos T;
  T.x0 = (t_begin % tiles_x) * WG_THREADS;
  T.y = (t_begin / tiles_x) % ny;
  T.b = t_begin / (tiles_x * ny);
  const float omega = p.omega;

  uint32_t phase = 0;
  bool fail = false;
  float db3[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) db3[i] = 0.f;

// leader waits for the warpgroup's last commit; the named barrier carries the verdict
#define WAIT_OR_BREAK()                                                  \
  if (leader) fail = !mbar_wait_bounded(bar, phase, WAIT_LIMIT);         \
  if (barrier_any(bar_id, WG_THREADS, fail)) break;                      \
  phase ^= 1;                                                            \
  fence_after_sync();
// all operand rows written: make them visible to the tensor core, then one thread issues
#define OPERANDS_READY()               \
  fence_proxy_async();                 \
  fence_before_sync();                 \
  named_barrier(bar_id, WG_THREADS);

  for (int it = 0; it < count; ++it) {
    const int x = T.x0 + r;
    const bool active = x < nx;
    const int ym = T.y == 0 ? ny - 1 : T.y - 1, yp = T.y == ny - 1 ? 0 : T.y + 1;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x >= nx - 1 ? 0 : x + 1;
    const float *gb = state + (size_t)T.b * Q * plane;
    float d[Q], pb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      d[i] = 0.f;
      pb[i] = 0.f;
    }
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
        const int ys = cy(i) == 0 ? T.y : (cy(i) == 1 ? ym : yp);
        d[i] = __ldg(gb + (size_t)i * plane + ys * nx + xs);
        pb[i] = __ldg(lam_next + (size_t)T.b * Q * plane + (size_t)i * plane + T.y * nx + x);
      }
    }
    // ---- forward recompute: moments, equilibrium, layer-1 operand
    const float drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    Moments m;
    m.drho = drho;
    m.rho = 1.0f + drho;
    const float inv_rho = 1.0f / m.rho;
    m.ux = jx * inv_rho;
    m.uy = jy * inv_rho;
    float deq[Q], xin[Q];
    shifted_feq(m, deq);
#pragma unroll
    for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * inv_rho;
    *reinterpret_cast<uint4 *>(B.a1 + canon_offset(r, 0, K1)) =
        make_uint4(pack_bf16x2(xin[0], xin[1]), pack_bf16x2(xin[2], xin[3]),
                   pack_bf16x2(xin[4], xin[5]), pack_bf16x2(xin[6], xin[7]));
    *reinterpret_cast<uint4 *>(B.a1 + canon_offset(r, 8, K1)) =
        make_uint4(pack_bf16x2(xin[8], 1.0f), 0u, 0u, 0u);
    OPERANDS_READY()
    if (leader) {
      fence_after_sync();
      mma_bf16(tm_wg + C_D, smem_desc(s_a1, 128, 16 * K1), smem_desc(s_w1, 128, 16 * K1), ID64, 0);
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    tanh_row(tm_row, B.h1, r, tm_wg + C_DH1 + lane_off);
    OPERANDS_READY()
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg + C_D, smem_desc(s_h1 + 256 * s, 128, 16 * K2),
                 smem_desc(s_w2 + 256 * s, 128, 16 * K2), ID64, s > 0);
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    tanh_row(tm_row, B.h2, r, tm_wg + C_DH2 + lane_off);
    OPERANDS_READY()
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg + C_D, smem_desc(s_h2 + 256 * s, 128, 16 * K2),
                 smem_desc(s_w3 + 256 * s, 128, 16 * K2), ID16, s > 0);
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    // ---- output of the network, then the reverse pass down to dL/do (FP32)
    float oh[Q];
    {
      uint32_t ov[16];
      tmem_ld16(tm_row, ov);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < Q; ++i) oh[i] = __uint_as_float(ov[i]);
      project9(oh);
    }
    // post = d + omega (deq - d) + rho omega ohat + fext(rho, u)
    float fb[Q], deqb[Q], ob[Q];
    float rhob = 0.f, uxb = 0.f, uyb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fb[i] = pb[i] * (1.0f - omega);
      deqb[i] = pb[i] * omega;
      ob[i] = m.rho * omega * pb[i];
      rhob = fmaf(omega * pb[i], oh[i], rhob);
    }
    if (p.force) {
      const float fx = __ldg(p.force + T.y);
      const float sxv = m.ux + fx * inv_rho;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float dr1, dx1, dy1, dr0, dx0, dy0;
        feq_partials(m.rho, sxv, m.uy, i, dr1, dx1, dy1);
        feq_partials(m.rho, m.ux, m.uy, i, dr0, dx0, dy0);
        rhob += pb[i] * ((dr1 - dx1 * fx * inv_rho * inv_rho) - dr0);
        uxb += pb[i] * (dx1 - dx0);
        uyb += pb[i] * (dy1 - dy0);
      }
    }
    project9(ob);  // dL/do = P dL/dohat (P symmetric)
#pragma unroll
    for (int i = 0; i < Q; ++i) db3[i] += ob[i];
    *reinterpret_cast<uint4 *>(B.ob + canon_offset(r, 0, 16)) =
        make_uint4(pack_bf16x2(ob[0], ob[1]), pack_bf16x2(ob[2], ob[3]),
                   pack_bf16x2(ob[4], ob[5]), pack_bf16x2(ob[6], ob[7]));
    *reinterpret_cast<uint4 *>(B.ob + canon_offset(r, 8, 16)) =
        make_uint4(pack_bf16x2(ob[8], 0.0f), 0u, 0u, 0u);
    OPERANDS_READY()
    if (leader) {  // dL/da2 (before the tanh derivative) = dL/do . W3
      fence_after_sync();
      mma_bf16(tm_wg + C_D, smem_desc(s_ob, 128, 256), smem_desc(s_w3t, 128, 256), ID64, 0);
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    dtanh_row(tm_row, tm_wg + C_DH2 + lane_off, B.a2b, r);
    OPERANDS_READY()
    if (leader) {  // dL/da1 (before the tanh derivative) = dL/da2 . W2
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_bf16(tm_wg + C_D, smem_desc(s_a2b + 256 * s, 128, 1024),
                 smem_desc(s_w2t + 256 * s, 128, 1024), ID64, s > 0);
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    dtanh_row(tm_row, tm_wg + C_DH1 + lane_off, B.a1b, r);
    OPERANDS_READY()
    if (leader) {
      fence_after_sync();
      // dL/dx = dL/da1 . W1
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_bf16(tm_wg + C_D, smem_desc(s_a1b + 256 * s, 128, 1024),
                 smem_desc(s_w1t + 256 * s, 128, 1024), ID16, s > 0);
      // weight gradients: reduction over the 128 nodes of the tile, 16 per MMA
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const uint32_t acc = (it > 0 || s > 0) ? 1u : 0u;
        mma_bf16(tm_wg + C_DW2, smem_desc(s_a2b + 2 * 1024 * s, 1024, 128),
                 smem_desc(s_h1 + 2 * 1280 * s, 1280, 128), IDW80, acc);
        mma_bf16(tm_wg + C_DW1, smem_desc(s_a1b + 2 * 1024 * s, 1024, 128),
                 smem_desc(s_a1 + 2 * 256 * s, 256, 128), IDW16, acc);
        mma_bf16(tm_wg + C_DW3, smem_desc(s_h2 + 2 * 1280 * s, 1280, 128),
                 smem_desc(s_ob + 2 * 256 * s, 256, 128), IDW16, acc);
      }
      mma_commit(bar);
    }
    WAIT_OR_BREAK()
    // ---- dL/dx -> rest of the chain rule (FP32), scatter lam to x - c_i
    {
      uint32_t xv[16];
      tmem_ld16(tm_row, xv);
      tmem_wait_ld();
      float xb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) xb[i] = __uint_as_float(xv[i]);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fb[i] += xb[i] * inv_rho;
        deqb[i] -= xb[i] * inv_rho;
        rhob -= xb[i] * xin[i] * inv_rho;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float dr, dux, duy;
        feq_partials(m.rho, m.ux, m.uy, i, dr, dux, duy);
        rhob = fmaf(deqb[i], dr, rhob);
        uxb = fmaf(deqb[i], dux, uxb);
        uyb = fmaf(deqb[i], duy, uyb);
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
#undef WAIT_OR_BREAK
#undef OPERANDS_READY

  if (leader && fail) {
    atomicOr(timeout_flag, 1);
    mbar_wait_bounded(bar, phase, WAIT_LIMIT);
  }
  // ---- this warpgroup's weight-gradient sums -> its row of partial sums
  float *row = partials + (size_t)gwg * NPARAMS;
  const bool have = count > 0 && !fail;
  {
    // db3: reduce the per-node sums of dL/do over the warpgroup
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v = db3[i];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if ((r & 31) == 0) S.db3[wg][warp_in_wg][i] = v;
    }
  }
  fence_after_sync();
  // M = 64 accumulators: row j lives in lane 32 (j / 16) + j % 16
  const int lane = r & 31;
  const int j = 16 * warp_in_wg + lane;
  uint32_t v2[80], v1[16], v3[16];
  tmem_ld32(tm_wg + C_DW2 + lane_off, *reinterpret_cast<uint32_t(*)[32]>(v2));
  tmem_ld32(tm_wg + C_DW2 + 32 + lane_off, *reinterpret_cast<uint32_t(*)[32]>(v2 + 32));
  tmem_ld16(tm_wg + C_DW2 + 64 + lane_off, *reinterpret_cast<uint32_t(*)[16]>(v2 + 64));
  tmem_ld16(tm_wg + C_DW1 + lane_off, v1);
  tmem_ld16(tm_wg + C_DW3 + lane_off, v3);
  tmem_wait_ld();
  named_barrier(bar_id, WG_THREADS);  // db3 partial sums visible
  if (lane < 16) {
    for (int k = 0; k < HIDDEN; ++k) {
      const float g = have ? __uint_as_float(v2[k]) : 0.f;
      float *dst = row + OFF_W2 + j * HIDDEN + k;
      *dst = accumulate ? *dst + g : g;
    }
    {
      const float g = have ? __uint_as_float(v2[64]) : 0.f;
      row[OFF_B2 + j] = accumulate ? row[OFF_B2 + j] + g : g;
    }
    for (int i = 0; i < 9; ++i) {
      const float g = have ? __uint_as_float(v1[i]) : 0.f;
      float *dst = row + OFF_W1 + j * 9 + i;
      *dst = accumulate ? *dst + g : g;
      const float g3 = have ? __uint_as_float(v3[i]) : 0.f;
      float *dst3 = row + OFF_W3 + i * HIDDEN + j;
      *dst3 = accumulate ? *dst3 + g3 : g3;
    }
    {
      const float g = have ? __uint_as_float(v1[9]) : 0.f;
      row[OFF_B1 + j] = accumulate ? row[OFF_B1 + j] + g : g;
    }
  }
  if (r < 9) {
    const float g = S.db3[wg][0][r] + S.db3[wg][1][r] + S.db3[wg][2][r] + S.db3[wg][3][r];
    row[OFF_B3 + r] = accumulate ? row[OFF_B3 + r] + g : g;
  }
  fence_before_sync();
  __syncthreads();
  if (tid < 32) tmem_dealloc(S.taddr, TMEM_COLS);
}

}  // namespace

int adjoint_tc_rows(const Grid &g, int sms) {
  const long long tiles = (long long)((g.nx + WG_THREADS - 1) / WG_THREADS) * g.ny * g.batch;
  long long ctas = (tiles + WGS - 1) / WGS;
  if (ctas > sms) ctas = sms;
  return (int)(ctas * WGS);
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
  k_adjoint_tc<<<rows / WGS, THREADS, SMEM_BYTES, s>>>(state_n, lam_next, lam_out, g.nx, g.ny,
                                                       g.batch, p, w, dw_partials, accumulate,
                                                       timeout_flag);
  return cudaGetLastError();
}

}  // namespace lbm
