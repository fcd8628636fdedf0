// mlp_bf16.cu -- fused pull-stream + learned collision with the MLP on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory).  Populations, moments, equilibrium, projection and the
// BGK/forcing update stay in FP32.
//
// Per node (Eq. S10-S12 with the network of this library):
//   x = (f - feq)/rho;  h1 = tanh(W1 x + b1);  h2 = tanh(W2 h1 + b2);  o = W3 h2 + b3
//   f' = f + (feq - f)/tau + (rho/tau) P o + f_ext,   P = mass/momentum projection
//
// Work decomposition.  A tile is 128 consecutive nodes of one row; one
// warpgroup (128 threads, thread r = node r = tensor-memory lane r) owns a
// tile at a time, and a CTA holds WGS warpgroups; every warpgroup walks its
// own contiguous range of tiles (persistent, grid = CTAS_PER_SM CTAs per SM).  Each layer is one GEMM with
// M = 128 nodes:
//   layer 1: [128 x 16] x [16 x 64]   K = 9 inputs + a constant-1 column (b1) + 6 zeros
//   layer 2: [128 x 80] x [80 x 64]   K = 64 hidden + constant-1 column (b2) + 15 zeros
//   layer 3: [128 x 80] x [80 x 16]   N = 9 outputs + 7 zero columns, b3 via the 1-column
// so the biases ride on the MMA.  Operands live in shared memory in the
// canonical K-major no-swizzle layout (umma.cuh); the accumulators of all
// three layers share the warpgroup's 64 tensor-memory columns (each layer's
// accumulator has been read back before the next GEMM is issued).  Between
// layers each thread reads its own row back with tcgen05.ld, rounds pairs to
// bf16x2 and applies the hardware tanh on the packed pairs, and writes the
// next operand row.  The populations of the next tile are loaded while the
// current tile's GEMMs run, and its layer-1 operand is written while the
// third GEMM runs (layer 1 has read its operand by then).
//
// Binding unit: the XU (MUFU) pipe.  Measured on this GPU with the
// epilogue's instruction mix (cvt + tanh.approx.bf16x2 per pair), the XU
// sustains ~0.24 tanh warp instructions per cycle per SM when 16 warps per SM
// feed it, so the 128 activations of a node cap the step near 37 G nodes/s
// however the GEMMs and memory traffic are scheduled (HBM alone would allow
// 94 G); with fewer warps in their tanh phase at once it reaches less.  Hence
// one CTA per SM of eight warpgroups (32 warps, 64 registers per thread; all
// 512 tensor-memory columns, 207 KB of shared memory): more warpgroups per SM
// keep more of them in their tanh epilogues at any time (measured at 4096^2:
// 4 warpgroups per SM 19.8 G nodes/s, 6: 23.6 G, 8: 24.3 G).  The tanh
// epilogue works through 16 columns at a time to stay within that register
// budget.
//
// Synchronisation per warpgroup: operand rows written by all 128 threads
// -> fence.proxy.async + named barrier -> one thread issues the MMAs and
// commits them to the warpgroup's mbarrier -> that thread alone polls the
// mbarrier (bounded) while the others sleep in a named barrier that also
// carries its verdict (bar.red.or), so a time-out is seen by the whole
// warpgroup at once: it leaves the loop, the leader sets the timeout flag and
// drains its outstanding commit, and tensor memory is freed.
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
#ifndef LBM_BF16_CTAS_PER_SM
#define LBM_BF16_CTAS_PER_SM 1
#endif
constexpr int WGS = LBM_BF16_WGS;                  // warpgroups per CTA
constexpr int CTAS_PER_SM = LBM_BF16_CTAS_PER_SM;  // resident CTAs per SM
constexpr int THREADS = WGS * WG_THREADS;
constexpr int K1 = 16, K2 = 80;        // padded K of layer 1 and of layers 2/3
// per CTA: 64 columns per warpgroup, rounded up to a power of two >= 32
constexpr uint32_t TMEM_COLS = WGS * 64 <= 64 ? 64 : (WGS * 64 <= 128 ? 128 : (WGS * 64 <= 256 ? 256 : 512));
#ifndef LBM_BF16_SLEEP_NS
#define LBM_BF16_SLEEP_NS 0
#endif
constexpr uint32_t WAIT_LIMIT = 1u << 20;  // polls; far above any real MMA latency
constexpr uint32_t SLEEP_NS = LBM_BF16_SLEEP_NS;  // suspend hint per poll (0: plain polls)

__device__ __forceinline__ bool wait_mma(uint32_t bar, uint32_t phase) {
  if (SLEEP_NS == 0) return mbar_wait_bounded(bar, phase, WAIT_LIMIT);
  return mbar_wait_sleep_bounded(bar, phase, WAIT_LIMIT / 64, SLEEP_NS);
}

struct __align__(1024) Smem {
  unsigned char w1[HIDDEN * K1 * 2];     // B of layer 1: [64 x 16]
  unsigned char w2[HIDDEN * K2 * 2];     // B of layer 2: [64 x 80]
  unsigned char w3[16 * K2 * 2];         // B of layer 3: [16 x 80]
  unsigned char a1[WGS][128 * K1 * 2];   // A of layer 1, per warpgroup
  unsigned char a23[WGS][128 * K2 * 2];  // A of layers 2 and 3, per warpgroup
  unsigned long long bar[WGS];
  uint32_t taddr;
};
// Shared memory requested per CTA: padded so that no more than CTAS_PER_SM
// CTAs share an SM (their tensor-memory allocations then always fit).
constexpr size_t SMEM_NEED = sizeof(Smem) + 1024;
constexpr size_t SMEM_FLOOR = (228 * 1024) / (CTAS_PER_SM + 1) + 1024;
constexpr size_t SMEM_BYTES = SMEM_NEED > SMEM_FLOOR ? SMEM_NEED : SMEM_FLOOR;
static_assert(SMEM_BYTES * CTAS_PER_SM <= 228 * 1024, "shared memory layout too large");
static_assert(CTAS_PER_SM * TMEM_COLS <= 512, "tensor memory oversubscribed");

__device__ __forceinline__ void store_bf16(unsigned char *base, int r, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + canon_offset(r, k, K)) = __float2bfloat16_rn(v);
}

template <int DTYPE>
__device__ __forceinline__ float wload(const void *p, int i) {
  if (DTYPE == 0) return __ldg(static_cast<const float *>(p) + i);
  return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
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

__device__ __forceinline__ void pull_node(const float *__restrict__ in, int plane, int nx,
                                          int ny, const TilePos &T, int x, float d[Q]) {
  const float *gb = in + (size_t)T.b * Q * plane;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = T.y == 0 ? ny - 1 : T.y - 1, yp = T.y == ny - 1 ? 0 : T.y + 1;
  const int r0 = T.y * nx, rm = ym * nx, rp = yp * nx;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
    const int rs = cy(i) == 0 ? r0 : (cy(i) == 1 ? rm : rp);
    d[i] = __ldg(gb + (size_t)i * plane + rs + xs);
  }
}

// Read the 64 accumulator columns of this thread's row, tanh on packed bf16
// pairs, write them as K columns 0..63 of the thread's layer-2/3 operand row.
__device__ __forceinline__ void tanh_row_to_operand(uint32_t tm_row, unsigned char *a23, int r) {
#pragma unroll
  for (int c = 0; c < HIDDEN; c += 16) {
    uint32_t v[16];
    tmem_ld16(tm_row + c, v);
    tmem_wait_ld();
    uint32_t p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      p[q] = tanh_bf16x2(pack_bf16x2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1])));
#pragma unroll
    for (int q = 0; q < 2; ++q)
      *reinterpret_cast<uint4 *>(a23 + canon_offset(r, c + 8 * q, K2)) =
          make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
  }
}

// Moments of shifted populations, reciprocal of rho rounded to nearest: the
// same arithmetic wherever a tile's moments are needed.
__device__ __forceinline__ Moments moments_rn(const float d[Q], float &inv_rho) {
  Moments m;
  m.drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
  const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
  const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
  m.rho = 1.0f + m.drho;
  inv_rho = __frcp_rn(m.rho);
  m.ux = jx * inv_rho;
  m.uy = jy * inv_rho;
  return m;
}

// x = (f - feq)/rho of this thread's node -> row r of the layer-1 operand (9
// inputs, the constant-1 bias column, zeros); flags an unstable node.
__device__ __forceinline__ void prep_x(const float d[Q], bool active, unsigned char *a1, int r,
                                       int *flag) {
  float inv_rho;
  const Moments m = moments_rn(d, inv_rho);
  flag_unstable(active && is_unstable(m), flag);
  float xin[Q];
  {
    float deq[Q];
    shifted_feq(m, deq);
#pragma unroll
    for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * inv_rho;
  }
  *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 0, K1)) =
      make_uint4(pack_bf16x2_alu(xin[0], xin[1]), pack_bf16x2_alu(xin[2], xin[3]),
                 pack_bf16x2_alu(xin[4], xin[5]), pack_bf16x2_alu(xin[6], xin[7]));
  *reinterpret_cast<uint4 *>(a1 + canon_offset(r, 8, K1)) =
      make_uint4(pack_bf16x2_alu(xin[8], 1.0f), 0u, 0u, 0u);
}

template <int DTYPE>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM)
    k_step_mlp_bf16(const float *__restrict__ in, float *__restrict__ out, int nx, int ny,
                    int batch, CollideParams p, const void *w1, const void *b1, const void *w2,
                    const void *b2, const void *w3, const void *b3, int *flag, int *timeout_flag) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int wg = tid / WG_THREADS;  // warpgroup within the CTA
  const int r = tid % WG_THREADS;   // row = node within the tile = TMEM lane
  const int warp_in_wg = r / 32;

  // ---- prologue: weights -> bf16 operand tiles, constant columns, barriers, TMEM
  for (int e = tid; e < HIDDEN * K1; e += THREADS) {
    const int n = e / K1, k = e % K1;
    const float v = k < 9 ? wload<DTYPE>(w1, n * 9 + k) : (k == 9 ? wload<DTYPE>(b1, n) : 0.f);
    store_bf16(S.w1, n, k, K1, v);
  }
  for (int e = tid; e < HIDDEN * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    const float v =
        k < HIDDEN ? wload<DTYPE>(w2, n * HIDDEN + k) : (k == HIDDEN ? wload<DTYPE>(b2, n) : 0.f);
    store_bf16(S.w2, n, k, K2, v);
  }
  for (int e = tid; e < 16 * K2; e += THREADS) {
    const int n = e / K2, k = e % K2;
    float v = 0.f;
    if (n < 9)
      v = k < HIDDEN ? wload<DTYPE>(w3, n * HIDDEN + k) : (k == HIDDEN ? wload<DTYPE>(b3, n) : 0.f);
    store_bf16(S.w3, n, k, K2, v);
  }
  // constant K columns 64..79 of this thread's layer-2/3 operand row: 1, 0, ..., 0
  {
    unsigned char *a23 = S.a23[wg];
    *reinterpret_cast<uint4 *>(a23 + canon_offset(r, 64, K2)) = make_uint4(0x3F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(a23 + canon_offset(r, 72, K2)) = make_uint4(0u, 0u, 0u, 0u);
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

  const uint32_t tm_wg = S.taddr + (uint32_t)(wg * 64);                // this WG's columns
  const uint32_t tm_row = tm_wg + ((uint32_t)(32 * warp_in_wg) << 16);  // + lane base
  const uint32_t bar = smem_u32(&S.bar[wg]);
  const uint32_t bar_id = 1 + wg;
  const bool leader = r == 0;
  unsigned char *a1 = S.a1[wg];
  unsigned char *a23 = S.a23[wg];
  const uint64_t da1 = smem_desc(smem_u32(a1), 128, 16 * K1);
  const uint64_t db1 = smem_desc(smem_u32(S.w1), 128, 16 * K1);
  const uint32_t sa23 = smem_u32(a23), sw2 = smem_u32(S.w2), sw3 = smem_u32(S.w3);
  constexpr uint32_t ID64 = idesc_bf16_f32(128, 64), ID16 = idesc_bf16_f32(128, 16);

  // ---- this warpgroup's contiguous range of tiles
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
  bool fail = false;  // the leader's last bounded wait gave up (leader only)

  float d[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = 0.f;
  if (count > 0 && T.x0 + r < nx) pull_node(in, plane, nx, ny, T, T.x0 + r, d);
  if (count > 0) prep_x(d, T.x0 + r < nx, a1, r, flag);

  for (int it = 0; it < count; ++it) {
    const int x = T.x0 + r;
    const bool active = x < nx;

    // ---- the tile's layer-1 operand rows are written (before the loop, or
    // during the previous tile's third GEMM)
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
      mma_bf16(tm_wg, da1, db1, ID64, 0);
      mma_commit(bar);
    }

    // ---- prefetch the next tile's populations while the GEMMs run
    TilePos N = T;
    N.advance(nx, ny);
    float dn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) dn[i] = 0.f;
    if (it + 1 < count && N.x0 + r < nx) pull_node(in, plane, nx, ny, N, N.x0 + r, dn);

    // ---- layer 1 epilogue: h1 = tanh(D1) -> operand of layer 2
    // (one thread polls the mbarrier; the others sleep in the named barrier)
    if (leader) fail = !wait_mma(bar, phase);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    phase ^= 1;
    fence_after_sync();
    tanh_row_to_operand(tm_row, a23, r);
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg, smem_desc(sa23 + 256 * s, 128, 16 * K2),
                 smem_desc(sw2 + 256 * s, 128, 16 * K2), ID64, s > 0);
      mma_commit(bar);
    }

    // ---- layer 2 epilogue: h2 = tanh(D2) -> operand of layer 3
    if (leader) fail = !wait_mma(bar, phase);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    phase ^= 1;
    fence_after_sync();
    tanh_row_to_operand(tm_row, a23, r);
    fence_proxy_async();
    fence_before_sync();
    named_barrier(bar_id, WG_THREADS);
    if (leader) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < K2 / 16; ++s)
        mma_bf16(tm_wg, smem_desc(sa23 + 256 * s, 128, 16 * K2),
                 smem_desc(sw3 + 256 * s, 128, 16 * K2), ID16, s > 0);
      mma_commit(bar);
    }

    // ---- the next tile's layer-1 operand while layer 3 runs (layer 1 of this
    // tile has completed, so a1 is free)
    if (it + 1 < count) prep_x(dn, N.x0 + r < nx, a1, r, flag);

    // ---- layer 3 epilogue: projection, BGK + learned correction + force, store
    if (leader) fail = !wait_mma(bar, phase);
    if (barrier_any(bar_id, WG_THREADS, fail)) break;
    {
      phase ^= 1;
      fence_after_sync();
      uint32_t ov[16];
      tmem_ld16(tm_row, ov);
      tmem_wait_ld();
      float o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) o[i] = __uint_as_float(ov[i]);
      project9(o);
      if (active) {
        float inv_rho;
        const Moments m = moments_rn(d, inv_rho);
        float deq[Q];
        shifted_feq(m, deq);
        const float rw = m.rho * omega;
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = fmaf(omega, deq[i] - d[i], d[i]) + rw * o[i];
        // EDM force (Eq. S5) for F = (fx, 0): the helper the BGK kernel uses,
        // so that a zero output layer reproduces BGK bit for bit
        if (p.force) add_edm_force_x(m, __ldg(p.force + T.y), d);
        float *ob = out + (size_t)T.b * Q * plane + T.y * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) ob[(size_t)i * plane] = d[i];
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = dn[i];
    T = N;
  }

  // the leader's wait gave up (the whole warpgroup left the loop together):
  // flag it and drain the outstanding commit (bounded) before tensor memory
  // is released
  if (leader && fail) {
    atomicOr(timeout_flag, 1);
    wait_mma(bar, phase);
  }
  fence_before_sync();
  __syncthreads();
  if (tid < 32) tmem_dealloc(S.taddr, TMEM_COLS);
}

}  // namespace

cudaError_t launch_step_mlp_bf16(const Grid &g, const float *in, float *out,
                                 const CollideParams &p, const void *const wp[6], int dtype,
                                 int *flag, int *timeout_flag, cudaStream_t s) {
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
  if ((long long)g.nx * g.ny * g.batch * Q >= (1LL << 31) || tiles >= (1LL << 31))
    return cudaErrorInvalidValue;  // 32-bit index arithmetic inside the kernel
  long long ctas = (tiles + WGS - 1) / WGS;
  if (ctas > (long long)CTAS_PER_SM * sms) ctas = (long long)CTAS_PER_SM * sms;
  kern<<<(unsigned)ctas, THREADS, SMEM_BYTES, s>>>(in, out, g.nx, g.ny, g.batch, p, wp[0], wp[1],
                                                   wp[2], wp[3], wp[4], wp[5], flag, timeout_flag);
  return cudaGetLastError();
}

}  // namespace lbm
