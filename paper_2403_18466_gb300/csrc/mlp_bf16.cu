// mlp_bf16.cu -- fused pull-stream + learned collision with the MLP on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory).  Populations, moments, equilibrium, projection and the
// BGK/forcing update stay in FP32.
//
// Per node (Eq. S10-S12 with the network of this library):
//   x = (f - feq)/rho;  h1 = tanh(W1 x + b1);  h2 = tanh(W2 h1 + b2);  o = W3 h2 + b3
//   f' = f + (feq - f)/tau + (rho/tau) P o + f_ext,   P = mass/momentum projection
//
// Work decomposition.  A tile is 128 consecutive nodes of one row; a
// warpgroup (128 threads, thread r = node r = tensor-memory lane r) owns one
// tile at a time and walks its own contiguous range of tiles; one persistent
// CTA per SM holds WGS = 8 warpgroups (1024 threads, 64 registers each, all
// 512 tensor-memory columns), so that many warps are in their activation
// epilogues at once.  Each layer is one GEMM with M = 128 nodes, BF16
// operands in shared memory (canonical K-major, no swizzle), FP32
// accumulators in the warpgroup's 64 tensor-memory columns:
//   layer 1: [128 x 16] x [16 x 64]   K = 9 inputs + a constant-1 column (b1) + 6 zeros
//   layer 2: [128 x 80] x [80 x 64]   K = 64 hidden + constant-1 column (b2) + 15 zeros
//   layer 3: [128 x 80] x [80 x 16]   N = 9 outputs + 7 zero columns, b3 via the 1-column
// so the biases ride on the MMA.  (Keeping the activations in tensor memory
// as the A operand instead needs 96 columns per tile, i.e. 5 tiles per SM; at
// that depth the GEMM round trips were no longer hidden: 21 G against 25 G
// nodes/s.)
//
// Between layers each thread reads its accumulator row with tcgen05.ld,
// applies tanh and writes the bf16 row of the next A operand to shared
// memory with 128-bit stores.  The activations are split between two units
// (TANH_XU_PAIRS of every 8 pairs of hidden units on the XU, the rest on the
// FMA pipe):
//   XU pairs:  cvt.rn.bf16x2.f32, then tanh.approx.bf16x2 (16.4 cycles of an
//     SM sub-partition per warp-wide pair, measured);
//   FMA pairs: the hidden units' weight rows and biases are pre-scaled by 1/4
//     (exact in bf16), so the accumulator holds y = a/4;  u = min(y^2, 1)
//     (fma.sat), tanh(a) ~ y P(u) with the degree-8 relative minimax
//     polynomial P of tanh(4 sqrt(u))/sqrt(u) on [0, 1] (odd in y, so small
//     activations keep their relative accuracy) in packed fma.rn.f32x2,
//     rounded to bf16 (cvt.rn) and clamped to [-1, 1] (min.xorsign.abs).
//     Maximum error before the rounding: 0.36 bf16 ulp of tanh (0.71 of the
//     half-ulp bar, checked on the GPU against tanhf); |a| >= 4 gives +-1,
//     which is the bf16 rounding of tanh(a) there.
// The FMA form takes ~26 cycles per warp-wide pair in isolation against 16.4
// for the XU form, and 13 issue slots against 2, so it pays only as a small
// share next to the kernel's other work (measured at 4096^2: 8 of 8 pairs on
// the XU 26.2 G nodes/s, 7 of 8: 26.5 G, 6: 25.8 G; 4 of 8, in an earlier
// form of the kernel: 20.3 G against 25.3 G for 7 of 8).
//
// Per node the moments, equilibrium, x and the BGK + force update are
// computed once, while the previous tile's last GEMM runs; the epilogue of
// layer 3 only projects o and adds (rho/tau) P o to the stored update.
//
// Synchronisation per warpgroup: operand rows written by all 128 threads ->
// fence.proxy.async + fence::before_thread_sync + named barrier -> one thread
// issues the MMAs and commits them to the warpgroup's mbarrier -> that thread
// alone polls the mbarrier (bounded) while the others sleep in a named
// barrier that also carries its verdict (bar.red.or), so a time-out is seen by
// the whole warpgroup at once: it leaves the loop, the leader sets the timeout
// flag and drains its outstanding commit (full limit), and tensor memory is
// always freed.
//
// Consecutive steps of one call are programmatic dependent launches: a step's
// prologue (weights to shared memory, tensor-memory allocation) runs on the
// SMs that the previous step has already left, and griddepcontrol.wait holds
// it back from the state buffers until that step has completed.
#include <cuda_bf16.h>

#include "kernels.h"
#include "lattice.cuh"
#include "umma.cuh"

namespace lbm {
namespace {

using namespace umma;

constexpr int WG_THREADS = 128;
#ifndef LBM_BF16_WGS
#define LBM_BF16_WGS 8
#endif
#ifndef LBM_TANH_XU_PAIRS
#define LBM_TANH_XU_PAIRS 7
#endif
#ifndef LBM_TANH_XU_FORM
#define LBM_TANH_XU_FORM 0
#endif
#ifndef LBM_TANH_FMA_PACK
#define LBM_TANH_FMA_PACK 0
#endif
constexpr int WGS = LBM_BF16_WGS;  // tile warpgroups per CTA (one CTA per SM)
// XU form: 0 = cvt.rn.bf16x2.f32 then tanh.approx.bf16x2 (20 XU cycles per
// warp-wide pair); 1 = tanh.approx.f32 on both FP32 values, packed to bf16 on
// the ALU (16 XU cycles per pair)
constexpr int XU_FORM = LBM_TANH_XU_FORM;
// bf16 packing of the FMA form: 0 = cvt.rn.bf16x2.f32 (XU), 1 = integer
// rounding on the ALU (ties away from zero)
constexpr int FMA_PACK = LBM_TANH_FMA_PACK;
#ifndef LBM_LEADER_SPREAD
#define LBM_LEADER_SPREAD 1
#endif
constexpr bool LEADER_SPREAD = LBM_LEADER_SPREAD != 0;
constexpr int THREADS = WGS * WG_THREADS;
constexpr int XU_PAIRS = LBM_TANH_XU_PAIRS;  // of every 8 activation pairs, on the XU
static_assert(XU_PAIRS >= 0 && XU_PAIRS <= 8, "split of 8 pairs");
constexpr int K1 = 16, K2 = 80;  // padded K of layer 1 and of layers 2/3
#ifndef LBM_EPI_COLS
#define LBM_EPI_COLS 16
#endif
// accumulator columns read per tensor-memory wait in the hidden epilogues
constexpr int EPI_COLS = LBM_EPI_COLS;
static_assert(EPI_COLS == 16 || EPI_COLS == 32, "16 or 32 columns per read");
// tensor memory: 64 accumulator columns per warpgroup
constexpr uint32_t TMEM_COLS = 512;
static_assert(WGS * 64 <= (int)TMEM_COLS, "tensor memory layout");
constexpr uint32_t DEFAULT_WAIT_LIMIT = 1u << 20;  // polls; far above any real MMA latency

// Bounded wait for a GEMM's commit.  A limit of 1024 polls or more uses
// mbarrier.try_wait (the thread is suspended until the phase completes or a
// short system time limit passes); a smaller limit polls with the
// non-blocking test_wait, so that it runs out after that many polls -- the
// way a test makes a wait give up.
__device__ __forceinline__ bool wait_gemm(uint32_t bar, uint32_t phase, uint32_t limit) {
  if (limit >= 1024) return mbar_wait_bounded(bar, phase, limit);
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_test_wait(bar, phase)) return true;
  return false;
}

// Degree-8 relative minimax polynomial of tanh(4 sqrt(u)) / sqrt(u) on [0, 1]
// (Lawson-weighted least squares, monomial basis, coefficients rounded to
// float32); tanh(4y) ~ y P(y^2) for |y| <= 1.
constexpr float TP0 = 3.9946699142456055f, TP1 = -20.35879898071289f, TP2 = 103.5002670288086f,
                TP3 = -381.81884765625f, TP4 = 933.0108642578125f, TP5 = -1447.415283203125f,
                TP6 = 1361.048095703125f, TP7 = -704.948486328125f, TP8 = 153.9882049560547f;

// True if hidden unit n is evaluated on the FMA pipe (its pre-activation is
// then accumulated pre-scaled by 1/4).
__host__ __device__ constexpr bool fma_unit(int n) { return (n % 16) >= 2 * XU_PAIRS; }

struct __align__(1024) Smem {
  unsigned char w1[HIDDEN * K1 * 2];     // B of layer 1: [64 x 16] = W1 | b1 | 0
  unsigned char w2[HIDDEN * K2 * 2];     // B of layer 2: [64 x 80] = W2 | b2 | 0
  unsigned char w3[16 * K2 * 2];         // B of layer 3: [16 x 80] = W3 | b3 | 0, rows 9..15 zero
  unsigned char a1[WGS][128 * K1 * 2];   // A of layer 1, per warpgroup
  unsigned char a23[WGS][128 * K2 * 2];  // A of layers 2 and 3, per warpgroup
  unsigned long long bar[WGS];
  uint32_t taddr;
};
// One CTA per SM (its tensor-memory allocation takes all 512 columns): the
// dynamic shared memory request is padded so that no second CTA fits.
constexpr size_t SMEM_BYTES = (sizeof(Smem) + 1024) > 120 * 1024 ? sizeof(Smem) + 1024 : 120 * 1024;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory layout too large");

__device__ __forceinline__ void store_bf16(unsigned char *base, int r, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + canon_offset(r, k, K)) = __float2bfloat16_rn(v);
}

template <int DTYPE>
__device__ __forceinline__ float wload(const void *p, int i) {
  if (DTYPE == 0) return __ldg(static_cast<const float *>(p) + i);
  return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}

// ---- activations ---------------------------------------------------------
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float sat_sq(float y) {
  float u;
  asm("fma.rn.sat.f32 %0, %1, %1, 0f00000000;" : "=f"(u) : "f"(y));
  return u;
}
__device__ __forceinline__ uint32_t clamp_unit_bf16x2(uint32_t v) {
  uint32_t r;
  asm("min.xorsign.abs.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0x3F803F80u));
  return r;
}
__device__ __forceinline__ float tanh_f32(float a) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
// XU pair: hardware tanh (see XU_FORM).
__device__ __forceinline__ uint32_t act_xu(float a0, float a1) {
  if (XU_FORM == 1) return pack_bf16x2_alu(tanh_f32(a0), tanh_f32(a1));
  return tanh_bf16x2(pack_bf16x2(a0, a1));
}
// FMA pair: y0, y1 = a/4 of the two units; tanh(a) ~ y P(min(y^2, 1)).
__device__ __forceinline__ uint32_t act_fma(float y0, float y1) {
  const uint64_t u = f2(sat_sq(y0), sat_sq(y1));
  uint64_t q = fma2(f2(TP8, TP8), u, f2(TP7, TP7));
  q = fma2(q, u, f2(TP6, TP6));
  q = fma2(q, u, f2(TP5, TP5));
  q = fma2(q, u, f2(TP4, TP4));
  q = fma2(q, u, f2(TP3, TP3));
  q = fma2(q, u, f2(TP2, TP2));
  q = fma2(q, u, f2(TP1, TP1));
  q = fma2(q, u, f2(TP0, TP0));
  const uint64_t h = mul2(f2(y0, y1), q);
  const float h0 = __uint_as_float((uint32_t)h), h1 = __uint_as_float((uint32_t)(h >> 32));
  return clamp_unit_bf16x2(FMA_PACK == 1 ? pack_bf16x2_alu(h0, h1) : pack_bf16x2(h0, h1));
}

// Accumulator columns [0, 64) of this thread's row -> tanh -> bf16 pairs as
// K columns 0..63 of row r of the layer-2/3 operand (16 columns at a time,
// within the 64-register budget).
__device__ __forceinline__ void hidden_epilogue(uint32_t tm_row, unsigned char *a23, int r) {
#pragma unroll
  for (int c = 0; c < HIDDEN; c += EPI_COLS) {
    uint32_t v[EPI_COLS];
    if (EPI_COLS == 32) tmem_ld32(tm_row + c, *reinterpret_cast<uint32_t(*)[32]>(v));
    else tmem_ld16(tm_row + c, *reinterpret_cast<uint32_t(*)[16]>(v));
    tmem_wait_ld();
    uint32_t p[EPI_COLS / 2];
#pragma unroll
    for (int q = 0; q < EPI_COLS / 2; ++q) {
      const float a0 = __uint_as_float(v[2 * q]), a1 = __uint_as_float(v[2 * q + 1]);
      p[q] = fma_unit(c + 2 * q) ? act_fma(a0, a1) : act_xu(a0, a1);
    }
#pragma unroll
    for (int q = 0; q < EPI_COLS / 8; ++q)
      *reinterpret_cast<uint4 *>(a23 + canon_offset(r, c + 8 * q, K2)) =
          make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
  }
}

// Position of a tile: lattice b, row y, first column x0.  Walked incrementally.
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

// Pre-collision populations (shifted) of node x of tile T: pull from the
// upstream neighbours with periodic wrap.
__device__ __forceinline__ void pull_node(const float *__restrict__ in, size_t plane, int nx,
                                          int ny, const TilePos &T, int x, float d[Q]) {
  const float *gb = in + (size_t)T.b * Q * plane;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = T.y == 0 ? ny - 1 : T.y - 1, yp = T.y == ny - 1 ? 0 : T.y + 1;
  const size_t r0 = (size_t)T.y * nx, rm = (size_t)ym * nx, rp = (size_t)yp * nx;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
    const size_t rs = cy(i) == 0 ? r0 : (cy(i) == 1 ? rm : rp);
    d[i] = __ldg(gb + (size_t)i * plane + rs + xs);
  }
}

// Everything of a node's update that does not need the network: moments,
// x = (f - feq)/rho written as row r of the layer-1 operand (9 inputs, the
// constant-1 bias column, zeros; bf16 with integer rounding on the ALU), the
// BGK + force update (the same helpers as the BGK kernel, so a zero output
// layer reproduces BGK bit for bit; fx = 0 on a lattice without forcing, so
// there is no branch) and rho/tau.  Returns true for an unstable node.
struct NodePrep {
  float base[Q];
  float rw;
};
__device__ __forceinline__ bool prep_node(const float d[Q], float omega, float fx,
                                          unsigned char *a1, int r, NodePrep &P) {
  const Moments m = node_moments(d);
  float deq[Q];
  shifted_feq(m, deq);
  float xin[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * m.inv_rho;
  *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 0, K1)) =
      make_uint4(pack_bf16x2_alu(xin[0], xin[1]), pack_bf16x2_alu(xin[2], xin[3]),
                 pack_bf16x2_alu(xin[4], xin[5]), pack_bf16x2_alu(xin[6], xin[7]));
  *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 8, K1)) =
      make_uint4(pack_bf16x2_alu(xin[8], 1.0f), 0u, 0u, 0u);
#pragma unroll
  for (int i = 0; i < Q; ++i) P.base[i] = bgk_relax(d[i], deq[i], omega);
  add_edm_force_x(m, fx, P.base);
  P.rw = m.rho * omega;
  return is_unstable(m);
}

// f' = base + (rho/tau) P o, with P the projection removing span{1, c_x, c_y}
// (Eqs. S11-S12: kappa_1 = -sum o / 9, kappa_a = -sum o c_a / 6 for D2Q9).
__device__ __forceinline__ void finish_node(const uint32_t ov[16], const NodePrep &P,
                                            float out[Q]) {
  float o[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) o[i] = __uint_as_float(ov[i]);
  const float s = ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7])) + o[8];
  const float sx = (o[1] - o[3]) + (o[5] - o[6]) + (o[8] - o[7]);
  const float sy = (o[2] - o[4]) + (o[5] + o[6]) - (o[7] + o[8]);
  const float k1 = -s * (1.0f / 9.0f), k2 = -sx * (1.0f / 6.0f), k3 = -sy * (1.0f / 6.0f);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float oi = o[i] + (k1 + ((float)cx(i) * k2 + (float)cy(i) * k3));
    out[i] = fmaf(P.rw, oi, P.base[i]);
  }
}

template <int DTYPE>
__global__ void __launch_bounds__(THREADS, 1)
    k_step_mlp_bf16(const float *__restrict__ in, float *__restrict__ out, int nx, int ny,
                    int batch, CollideParams p, const void *w1, const void *b1, const void *w2,
                    const void *b2, const void *w3, const void *b3, int *flag, int *timeout_flag,
                    uint32_t wait_limit) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int wg = tid / WG_THREADS;  // warpgroup within the CTA
  const int r = tid % WG_THREADS;   // row = node within the tile = TMEM lane
  const int warp_in_wg = r / 32;

  // ---- prologue: weights -> bf16 operand tiles (FMA-form units pre-scaled
  // by 1/4, exact in bf16), constant columns, barriers, tensor memory
  for (int e = tid; e < HIDDEN * K1; e += THREADS) {
    const int n = e / K1, k = e % K1;
    float v = k < 9 ? wload<DTYPE>(w1, n * 9 + k) : (k == 9 ? wload<DTYPE>(b1, n) : 0.f);
    if (fma_unit(n)) v *= 0.25f;
    store_bf16(S.w1, n, k, K1, v);
  }
  for (int e = tid; e < HIDDEN * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    float v = k < HIDDEN ? wload<DTYPE>(w2, n * HIDDEN + k) : (k == HIDDEN ? wload<DTYPE>(b2, n) : 0.f);
    if (fma_unit(n)) v *= 0.25f;
    store_bf16(S.w2, n, k, K2, v);
  }
  for (int e = tid; e < 16 * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    float v = 0.f;
    if (n < 9)
      v = k < HIDDEN ? wload<DTYPE>(w3, n * HIDDEN + k) : (k == HIDDEN ? wload<DTYPE>(b3, n) : 0.f);
    store_bf16(S.w3, n, k, K2, v);
  }
  unsigned char *a1 = S.a1[wg];
  unsigned char *a23 = S.a23[wg];
  // constant K columns 64..79 of this thread's layer-2/3 operand row: 1, 0, ..., 0
  *reinterpret_cast<uint4 *>(a23 + canon_offset(r, 64, K2)) = make_uint4(0x3F80u, 0u, 0u, 0u);
  *reinterpret_cast<uint4 *>(a23 + canon_offset(r, 72, K2)) = make_uint4(0u, 0u, 0u, 0u);
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

  const uint32_t tm_wg = S.taddr + (uint32_t)(wg * 64);                // this WG's columns
  const uint32_t tm_row = tm_wg + ((uint32_t)(32 * warp_in_wg) << 16);  // + lane base
  const uint32_t bar = smem_u32(&S.bar[wg]);
  const uint32_t bar_id = 1 + wg;
  // the thread that issues and waits for the warpgroup's GEMMs: lane 0 of
  // warp (wg mod 4) of the warpgroup, so that the eight leaders sit on all
  // four SM sub-partitions (CTA warp w runs on sub-partition w mod 4)
  const bool leader = LEADER_SPREAD ? r == 32 * (wg & 3) : r == 0;
  // operand descriptors; a K = 16 slice further is 256 bytes = 16 units of the
  // descriptor's start-address field (shared addresses stay below 2^18, so
  // the 14-bit field does not overflow)
  const uint64_t da1 = smem_desc(smem_u32(a1), 128, 16 * K1);
  const uint64_t db1 = smem_desc(smem_u32(S.w1), 128, 16 * K1);
  const uint64_t d23 = smem_desc(smem_u32(a23), 128, 16 * K2);
  const uint64_t dw2 = smem_desc(smem_u32(S.w2), 128, 16 * K2);
  const uint64_t dw3 = smem_desc(smem_u32(S.w3), 128, 16 * K2);
  constexpr uint32_t ID64 = idesc_bf16_f32(128, 64), ID16 = idesc_bf16_f32(128, 16);

  // ---- this warpgroup's contiguous range of tiles
  const size_t plane = (size_t)nx * ny;
  const int tiles_x = (nx + WG_THREADS - 1) / WG_THREADS;
  const long long ntiles = (long long)tiles_x * ny * batch;
  const long long nwg = (long long)gridDim.x * WGS;
  const long long gwg = (long long)blockIdx.x * WGS + wg;
  const long long per = ntiles / nwg, extra = ntiles % nwg;
  const long long t_begin = gwg * per + (gwg < extra ? gwg : extra);
  const int count = (int)(per + (gwg < extra ? 1 : 0));
  TilePos T;
  T.x0 = (int)(t_begin % tiles_x) * WG_THREADS;
  T.y = (int)((t_begin / tiles_x) % ny);
  T.b = (int)(t_begin / ((long long)tiles_x * ny));
  const float omega = p.omega;

  // Everything above reads only the weights.  With programmatic dependent
  // launch this CTA may be running while the previous step (which writes `in`
  // and reads `out`) finishes on other SMs: wait for it before the first
  // access to either state buffer, and let the next step start its own
  // prologue as SMs free up (a CTA holds all of an SM's registers, so the
  // next step's CTA becomes resident only after this one exits).
  griddep_wait();
  griddep_launch_dependents();

  uint32_t phase = 0;
  bool fail = false;  // the leader's last bounded wait gave up (leader only)
  bool bad = false;   // an unstable node was met (per thread)

  NodePrep P;
  {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = 0.f;
    const bool act = count > 0 && T.x0 + r < nx;
    if (act) pull_node(in, plane, nx, ny, T, T.x0 + r, d);
    const bool b0 =
        prep_node(d, omega, (count > 0 && p.force) ? __ldg(p.force + T.y) : 0.f, a1, r, P);
    bad = act && b0;
  }

  for (int it = 0; it < count; ++it) {
    const int x = T.x0 + r;
    const bool active = x < nx;

    // ---- layer 1 (its operand rows were written before the loop or during
    // the previous tile's layer 3)
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
      mma_bf16(tm_wg, da1, db1, ID64, 0);
      mma_commit(bar);
    }

    // ---- prefetch the next tile's populations and force while the GEMMs run
    TilePos N = T;
    N.advance(nx, ny);
    const bool more = it + 1 < count;
    const bool nact = more && N.x0 + r < nx;
    float dn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) dn[i] = 0.f;
    if (nact) pull_node(in, plane, nx, ny, N, N.x0 + r, dn);
    const float fxn = (more && p.force) ? __ldg(p.force + N.y) : 0.f;

    // ---- layer 1 epilogue: h1 -> operand of layer 2; layer 2
    if (leader) fail = !wait_gemm(bar, phase, wait_limit);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    phase ^= 1;
    fence_after_sync();
    hidden_epilogue(tm_row, a23, r);
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg, d23 + 16 * s, dw2 + 16 * s, ID64, s > 0);
      mma_commit(bar);
    }

    // ---- layer 2 epilogue: h2 -> operand of layer 3; layer 3
    if (leader) fail = !wait_gemm(bar, phase, wait_limit);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    phase ^= 1;
    fence_after_sync();
    hidden_epilogue(tm_row, a23, r);
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg, d23 + 16 * s, dw3 + 16 * s, ID16, s > 0);
      mma_commit(bar);
    }

    // ---- the next tile's per-node work while layer 3 runs (layer 1 of this
    // tile has read a1)
    NodePrep Pn;
    {
      const bool bn = prep_node(dn, omega, fxn, a1, r, Pn);
      bad |= nact && bn;
    }

    // ---- layer 3 epilogue: projection, update, store
    if (leader) fail = !wait_gemm(bar, phase, wait_limit);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    phase ^= 1;
    fence_after_sync();
    {
      uint32_t ov[16];
      tmem_ld16(tm_row, ov);
      tmem_wait_ld();
      if (active) {
        float f[Q];
        finish_node(ov, P, f);
        float *ob = out + (size_t)T.b * Q * plane + (size_t)T.y * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) ob[(size_t)i * plane] = f[i];
      }
    }
    P = Pn;
    T = N;
  }

  // the leader's wait gave up (the whole warpgroup left the loop together):
  // flag it and drain the outstanding commit (full limit) before tensor
  // memory is released
  if (leader && fail) {
    atomicOr(timeout_flag, 1);
    mbar_wait_bounded(bar, phase, DEFAULT_WAIT_LIMIT);
  }
  flag_unstable(bad, flag);
  fence_before_sync();
  __syncthreads();
  if (tid < 32) tmem_dealloc(S.taddr, TMEM_COLS);
}

// The activations of the step kernel applied element-wise (path 0: XU pair,
// 1: FMA pair as stored, 2: FMA pair before its bf16 rounding), for tests of
// their accuracy against tanh.  Odd counts: the last pair repeats its input.
__global__ void k_activation(const float *__restrict__ a, int n, int path, float *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * j >= n) return;
  const float a0 = a[2 * j], a1 = 2 * j + 1 < n ? a[2 * j + 1] : a0;
  float r0, r1;
  if (path == 2) {
    const float y0 = 0.25f * a0, y1 = 0.25f * a1;
    const uint64_t u = f2(sat_sq(y0), sat_sq(y1));
    uint64_t q = fma2(f2(TP8, TP8), u, f2(TP7, TP7));
    q = fma2(q, u, f2(TP6, TP6));
    q = fma2(q, u, f2(TP5, TP5));
    q = fma2(q, u, f2(TP4, TP4));
    q = fma2(q, u, f2(TP3, TP3));
    q = fma2(q, u, f2(TP2, TP2));
    q = fma2(q, u, f2(TP1, TP1));
    q = fma2(q, u, f2(TP0, TP0));
    const uint64_t h = mul2(f2(y0, y1), q);
    r0 = fminf(fmaxf(__uint_as_float((uint32_t)h), -1.0f), 1.0f);
    r1 = fminf(fmaxf(__uint_as_float((uint32_t)(h >> 32)), -1.0f), 1.0f);
  } else {
    const uint32_t v = path == 0 ? act_xu(a0, a1) : act_fma(0.25f * a0, 0.25f * a1);
    r0 = __uint_as_float(v << 16);
    r1 = __uint_as_float(v & 0xffff0000u);
  }
  out[2 * j] = r0;
  if (2 * j + 1 < n) out[2 * j + 1] = r1;
}

}  // namespace

void mlp_bf16_layout(int *warpgroups, int *xu_pairs_per_8) {
  if (warpgroups) *warpgroups = WGS;
  if (xu_pairs_per_8) *xu_pairs_per_8 = XU_PAIRS;
}

cudaError_t launch_activation(const float *a, int n, int path, float *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int pairs = (n + 1) / 2;
  k_activation<<<(pairs + 255) / 256, 256, 0, s>>>(a, n, path, out);
  return cudaGetLastError();
}

cudaError_t launch_step_mlp_bf16(const Grid &g, const float *in, float *out,
                                 const CollideParams &p, const void *const wp[6], int dtype,
                                 int *flag, int *timeout_flag, cudaStream_t s,
                                 unsigned wait_limit, int max_ctas, bool chain) {
  static int sms = 0;
  static bool attr_done[2] = {false, false};
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  auto kern = dtype == 0 ? k_step_mlp_bf16<0> : k_step_mlp_bf16<1>;
  if (!attr_done[dtype]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_done[dtype] = true;
  }
  const long long tiles = (long long)((g.nx + WG_THREADS - 1) / WG_THREADS) * g.ny * g.batch;
  long long ctas = (tiles + WGS - 1) / WGS;
  if (ctas > (long long)sms) ctas = sms;
  if (max_ctas > 0 && ctas > max_ctas) ctas = max_ctas;
  if (wait_limit == 0) wait_limit = DEFAULT_WAIT_LIMIT;
  // programmatic dependent launch after a step of this kernel (the prologue --
  // weights to shared memory, tensor-memory allocation -- overlaps that step's
  // last tiles); otherwise plain stream order, since the prologue reads the
  // weights, which an earlier operation may still be writing
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chain ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, in, out, g.nx, g.ny, g.batch, p, wp[0], wp[1], wp[2],
                            wp[3], wp[4], wp[5], flag, timeout_flag, wait_limit);
}

}  // namespace lbm
