// d3q19_mlp_tc.cu -- the paper's learned collision on D3Q19 with its network
// (19 -> 300 -> 300 -> 100 -> 19, LeakyReLU, conservation layer with kappa
// denominators 19 and 10) on the 5th-generation tensor cores: tcgen05 MMAs with
// BF16 operands and FP32 accumulation in tensor memory, fused with the pull-
// stream, the BGK update and the EDM forcing (populations stay FP32).
//
// Per node: x = (f - feq)/rho; h1 = lrelu(W1 x + b1); h2 = lrelu(W2 h1 + b2);
// h3 = lrelu(W3 h2 + b3); o = W4 h3 + b4; f' = f + (feq - f)/tau + (rho/tau) P o + f_ext.
//
// GEMMs per tile of M = 128 nodes (one x row segment), biases folded in as a
// constant-1 operand column:
//   L1  [128 x  32] x [ 32 x 304]   K = 19 inputs + 1 + 12 zeros; N = 300 + 4 zero rows
//   L2  [128 x 304] x [304 x 304]   K = 300 + 1 + 3 zeros
//   L3  [128 x 304] x [304 x 112]   N = 100 + 12 zero rows
//   L4  [128 x 112] x [112 x  32]   K = 100 + 1 + 11 zeros; N = 19 + 13 zero rows
// N = 304 exceeds one MMA, so L1 and L2 issue two MMAs per K step (N = 160, 144).
//
// The paper's network has 280 KB of BF16 weights, more than an SM's shared
// memory, so W1 and W4 stay resident and W2 and W3 are streamed every tile in
// K chunks of 32 (19,456 / 7,168 bytes) through a 6-slot ring filled by bulk
// copies (cp.async.bulk) from a pre-laid-out copy in global memory (the L2
// cache holds it).  The activations are the A operand in shared memory in the
// canonical K-major layout of umma.cuh; the accumulator uses up to 304 tensor-
// memory columns.
//
// Roles in a CTA of 320 threads (one CTA per SM, persistent over a contiguous
// range of tiles):
//   warps 0-3  (WG0)  node work of the tile (pull, moments, x, final update,
//                     store) and the epilogue of the low accumulator columns;
//   warps 4-7  (WG1)  epilogue of the high accumulator columns;
//   warp 8            MMA issue (one thread);
//   warp 9            weight-ring producer (one thread).
// Hand-offs are mbarriers: x ready (128 arrivals), A ready (256 arrivals), the
// accumulator ready (an MMA commit), and the ring's full/empty pairs.  Every
// wait is bounded; on a time-out the kernel records it in shared memory, all
// roles leave their loops, in-flight copies and MMAs are drained with bounded
// waits, the tensor memory is freed and the timeout flag is set.
#include <cuda_bf16.h>

#include "d3q19.cuh"
#include "kernels3d.h"
#include "umma.cuh"

namespace lbm {
namespace d3 {
namespace {

using namespace umma;

constexpr int KX = 32;     // layer-1 K
constexpr int NH = 304;    // padded hidden width (rows of W1, W2 as B operands)
constexpr int KH = 304;    // K of layers 2 and 3
constexpr int N3 = 112;    // rows of W3
constexpr int K4 = 112;    // K of layer 4
constexpr int N4 = 32;     // rows of W4
constexpr int KC = 32;     // K per streamed chunk
constexpr int NCHUNK = 10; // 9 chunks of 32 + 1 of 16 per streamed matrix
constexpr int SLOTS = 6;
constexpr int SLOT_BYTES = NH * KC * 2;  // 19,456
constexpr int W1_BYTES = NH * KX * 2;    // 19,456
constexpr int W4_BYTES = N4 * K4 * 2;    // 7,168
constexpr int W2_CHUNK = NH * KC * 2;    // 19,456 (the last chunk uses half)
constexpr int W3_CHUNK = N3 * KC * 2;    // 7,168 (the last chunk uses half)
// pre-laid-out weights in global memory (bytes)
constexpr int G_W1 = 0;
constexpr int G_W4 = G_W1 + W1_BYTES;
constexpr int G_W2 = G_W4 + W4_BYTES;
constexpr int G_W3 = G_W2 + NCHUNK * W2_CHUNK;
constexpr int G_BYTES = G_W3 + NCHUNK * W3_CHUNK;  // 292,864

constexpr int THREADS = 320;
constexpr int MMA_WARP = 8, PROD_WARP = 9;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct __align__(1024) Smem {
  unsigned char w1[W1_BYTES];
  unsigned char w4[W4_BYTES];
  unsigned char x[128 * KX * 2];
  unsigned char a[128 * KH * 2];
  unsigned char ring[SLOTS][SLOT_BYTES];
  unsigned long long full[SLOTS], empty[SLOTS];
  unsigned long long xready, aready, accready, drain;
  uint32_t taddr;
  int err;
};
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;
static_assert(SMEM_BYTES <= 232448, "shared memory layout too large");

__host__ __device__ constexpr int chunk_k(int c) { return c < NCHUNK - 1 ? KC : KH - KC * (NCHUNK - 1); }

// ---- helpers ------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Bounded wait that also gives up early once another role has recorded an error.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, volatile int *err) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *err) return false;
  }
  atomicOr(const_cast<int *>(err), 1);
  return false;
}
// The same for a whole warp: lane 0 polls, the verdict is broadcast, so the
// warp stays converged for the .sync.aligned tensor-memory loads that follow.
__device__ __forceinline__ bool wait_phase_warp(uint32_t bar, uint32_t parity, volatile int *err) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = wait_phase(bar, parity, err);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint64_t a, uint64_t b, uint32_t id, bool acc) {
  mma_bf16(d, a, b, id, acc ? 1u : 0u);
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) { return pack_bf16x2(lo, hi); }
__device__ __forceinline__ float lrelu(float v) { return fmaxf(v, LEAKY * v); }

// Tile walk: 128 consecutive x of row (b, z, y).
struct Tile {
  int b, z, y, x0;
  __device__ __forceinline__ void set(int t, int tiles_x, int ny, int nz) {
    x0 = (t % tiles_x) * 128;
    int row = t / tiles_x;
    y = row % ny;
    row /= ny;
    z = row % nz;
    b = row / nz;
  }
};

__device__ __forceinline__ void pull19(const float *__restrict__ in, const Grid3 &g, const Tile &T,
                                       int x, float d[Q]) {
  const size_t vol = g.volume();
  const float *gb = in + (size_t)T.b * Q * vol;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int xs = x - cx(i), ys = T.y - cy(i), zs = T.z - cz(i);
    xs = xs < 0 ? xs + g.nx : (xs >= g.nx ? xs - g.nx : xs);
    ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
    zs = zs < 0 ? zs + g.nz : (zs >= g.nz ? zs - g.nz : zs);
    d[i] = __ldg(gb + (size_t)i * vol + ((size_t)zs * g.ny + ys) * g.nx + xs);
  }
}

// Drain accumulator columns [c0, c1) (multiples of 16) of this thread's row:
// LeakyReLU, bf16, into K columns of the A operand row r (row length KH).
// Columns at or above `kvalid` are not activations: `kvalid` gets the constant
// 1 (the bias column) and the rest zero.
__device__ __forceinline__ void drain_to_a(uint32_t tm_row, int c0, int c1, int kvalid,
                                           unsigned char *a, int r) {
  for (int c = c0; c < c1; c += 16) {
    uint32_t v[16];
    tmem_ld16(tm_row + (uint32_t)c, v);
    tmem_wait_ld();
    float h[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int k = c + q;
      h[q] = k < kvalid ? lrelu(__uint_as_float(v[q])) : (k == kvalid ? 1.0f : 0.0f);
    }
    uint32_t p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = pack2(h[2 * q], h[2 * q + 1]);
    *reinterpret_cast<uint4 *>(a + canon_offset(r, c, KH)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4 *>(a + canon_offset(r, c + 8, KH)) = make_uint4(p[4], p[5], p[6], p[7]);
  }
}

__global__ void __launch_bounds__(THREADS, 1)
    k3_step_mlp_tc(const float *__restrict__ in, float *__restrict__ out, Grid3 g, Collide3 cp,
                   const unsigned char *__restrict__ gw, int *flag, int *timeout_flag) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *err = &S.err;

  // ---- prologue: resident weights, barriers, tensor memory
  {
    const uint4 *src1 = reinterpret_cast<const uint4 *>(gw + G_W1);
    uint4 *dst1 = reinterpret_cast<uint4 *>(S.w1);
    for (int e = tid; e < W1_BYTES / 16; e += THREADS) dst1[e] = src1[e];
    const uint4 *src4 = reinterpret_cast<const uint4 *>(gw + G_W4);
    uint4 *dst4 = reinterpret_cast<uint4 *>(S.w4);
    for (int e = tid; e < W4_BYTES / 16; e += THREADS) dst4[e] = src4[e];
  }
  if (tid == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(smem_u32(&S.full[s]), 1);
      mbar_init(smem_u32(&S.empty[s]), 1);
    }
    mbar_init(smem_u32(&S.xready), 128);
    mbar_init(smem_u32(&S.aready), 256);
    mbar_init(smem_u32(&S.accready), 1);
    mbar_init(smem_u32(&S.drain), 1);
    S.err = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&S.taddr), 512);
    tmem_relinquish();
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = S.taddr;

  // ---- this CTA's contiguous range of tiles
  const int tiles_x = (g.nx + 127) / 128;
  const long long ntiles_ll = (long long)tiles_x * g.ny * g.nz * g.batch;
  const int ntiles = (int)ntiles_ll;
  const int per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
  const int t_begin = blockIdx.x * per + min((int)blockIdx.x, extra);
  const int count = per + ((int)blockIdx.x < extra ? 1 : 0);

  if (warp == PROD_WARP) {
    // ---------------- weight-ring producer
    if (lane == 0) {
      uint32_t uses[SLOTS] = {0, 0, 0, 0, 0, 0};
      int slot = 0;
      bool ok = true;
      for (int t = 0; t < count && ok; ++t) {
        for (int mat = 0; mat < 2 && ok; ++mat) {
          for (int c = 0; c < NCHUNK; ++c) {
            const uint32_t full = smem_u32(&S.full[slot]), empty = smem_u32(&S.empty[slot]);
            if (uses[slot] > 0 && !wait_phase(empty, (uses[slot] - 1) & 1u, err)) {
              ok = false;
              break;
            }
            const int rows = mat == 0 ? NH : N3;
            const uint32_t bytes = (uint32_t)(rows * chunk_k(c) * 2);
            const unsigned char *src =
                gw + (mat == 0 ? G_W2 + c * W2_CHUNK : G_W3 + c * W3_CHUNK);
            mbar_arrive_expect_tx(full, bytes);
            bulk_g2s(smem_u32(S.ring[slot]), src, bytes, full);
            ++uses[slot];
            slot = slot + 1 == SLOTS ? 0 : slot + 1;
          }
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int s = 0; s < SLOTS; ++s)
        if (uses[s] > 0) {
          const uint32_t full = smem_u32(&S.full[s]);
          for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
            if (mbar_try_wait(full, (uses[s] - 1) & 1u)) break;
        }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue
    if (lane == 0) {
      const uint32_t sx = smem_u32(S.x), sa = smem_u32(S.a), sw1 = smem_u32(S.w1),
                     sw4 = smem_u32(S.w4);
      const uint32_t bar_acc = smem_u32(&S.accready);
      constexpr uint32_t ID160 = idesc_bf16_f32(128, 160), ID144 = idesc_bf16_f32(128, 144),
                         ID112 = idesc_bf16_f32(128, 112), ID32 = idesc_bf16_f32(128, 32);
      uint32_t px = 0, pa = 0;
      uint32_t uses[SLOTS] = {0, 0, 0, 0, 0, 0};
      int slot = 0;
      bool issued = false;
      for (int t = 0; t < count; ++t) {
        // L1: A = x (K 32), B = W1 resident
        if (!wait_phase(smem_u32(&S.xready), px, err)) break;
        px ^= 1;
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < KX / 16; ++s) {
          const uint64_t a = smem_desc(sx + 256 * s, 128, 16 * KX);
          mma_ts(tmem, a, smem_desc(sw1 + 256 * s, 128, 16 * KX), ID160, s > 0);
          mma_ts(tmem + 160, a, smem_desc(sw1 + 20 * 16 * KX + 256 * s, 128, 16 * KX), ID144,
                 s > 0);
        }
        mma_commit(bar_acc);
        issued = true;
        // L2 and L3: A = activations (K 304), B = streamed chunks
        bool ok = true;
        for (int mat = 0; mat < 2 && ok; ++mat) {
          if (!wait_phase(smem_u32(&S.aready), pa, err)) {
            ok = false;
            break;
          }
          pa ^= 1;
          fence_after_sync();
          for (int c = 0; c < NCHUNK; ++c) {
            if (!wait_phase(smem_u32(&S.full[slot]), uses[slot] & 1u, err)) {
              ok = false;
              break;
            }
            fence_after_sync();
            const int kc = chunk_k(c);
            const uint32_t sb = smem_u32(S.ring[slot]);
            for (int s = 0; s < kc / 16; ++s) {
              const uint64_t a = smem_desc(sa + 256 * (2 * c + s), 128, 16 * KH);
              const bool acc = c > 0 || s > 0;
              if (mat == 0) {
                mma_ts(tmem, a, smem_desc(sb + 256 * s, 128, 16 * kc), ID160, acc);
                mma_ts(tmem + 160, a, smem_desc(sb + 20 * 16 * kc + 256 * s, 128, 16 * kc),
                       ID144, acc);
              } else {
                mma_ts(tmem, a, smem_desc(sb + 256 * s, 128, 16 * kc), ID112, acc);
              }
            }
            mma_commit(smem_u32(&S.empty[slot]));
            ++uses[slot];
            slot = slot + 1 == SLOTS ? 0 : slot + 1;
          }
          if (ok) mma_commit(bar_acc);
        }
        if (!ok) break;
        // L4: A = h3 (K 112 of the activation rows), B = W4 resident
        if (!wait_phase(smem_u32(&S.aready), pa, err)) break;
        pa ^= 1;
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < K4 / 16; ++s)
          mma_ts(tmem, smem_desc(sa + 256 * s, 128, 16 * KH),
                 smem_desc(sw4 + 256 * s, 128, 16 * K4), ID32, s > 0);
        mma_commit(bar_acc);
      }
      // drain outstanding MMAs before the tensor memory is freed
      if (issued) {
        mma_commit(smem_u32(&S.drain));
        for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
          if (mbar_try_wait(smem_u32(&S.drain), 0)) break;
      }
    }
  } else {
    // ---------------- node and epilogue warpgroups
    const int wg = warp >> 2;          // 0 or 1
    const int r = tid & 127;           // tile row = tensor-memory lane
    const uint32_t tm_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t bar_acc = smem_u32(&S.accready), bar_a = smem_u32(&S.aready),
                   bar_x = smem_u32(&S.xready);
    uint32_t pacc = 0;
    Tile T;
    T.set(t_begin, tiles_x, g.ny, g.nz);
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = 0.f;
    if (wg == 0 && count > 0 && T.x0 + r < g.nx) pull19(in, g, T, T.x0 + r, d);
    const size_t vol = g.volume();

    for (int t = 0; t < count; ++t) {
      const int x = T.x0 + r;
      const bool active = x < g.nx;
      Moments m = {0.f, 1.f, 0.f, 0.f, 0.f};
      float deq[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) deq[i] = 0.f;
      float inv_rho = 1.f;
      if (wg == 0) {
        // x = (f - feq)/rho -> row r of the layer-1 operand (19 + bias + zeros)
        m = node_moments(d);
        inv_rho = 1.0f / m.rho;
        {
          // sticky instability flag: one atomic at most per warp
          const unsigned mask = __ballot_sync(0xffffffffu, active && is_unstable(m));
          if (mask && lane == (__ffs(mask) - 1) && *reinterpret_cast<volatile int *>(flag) == 0)
            atomicOr(flag, 1);
        }
        shifted_feq(m, deq);
        float xi[32];
#pragma unroll
        for (int i = 0; i < 32; ++i)
          xi[i] = i < Q ? (active ? (d[i] - deq[i]) * inv_rho : 0.f) : (i == Q ? 1.0f : 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4 *>(S.x + canon_offset(r, 8 * q, KX)) =
              make_uint4(pack2(xi[8 * q], xi[8 * q + 1]), pack2(xi[8 * q + 2], xi[8 * q + 3]),
                         pack2(xi[8 * q + 4], xi[8 * q + 5]), pack2(xi[8 * q + 6], xi[8 * q + 7]));
        fence_proxy_async();
        fence_before_sync();
        mbar_arrive(bar_x);
      }
      // prefetch the next tile's populations while the GEMMs run
      Tile N = T;
      float dn[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) dn[i] = 0.f;
      if (wg == 0 && t + 1 < count) {
        N.set(t_begin + t + 1, tiles_x, g.ny, g.nz);
        if (N.x0 + r < g.nx) pull19(in, g, N, N.x0 + r, dn);
      }
      // L1 -> h1, L2 -> h2 (N = 304: WG0 columns 0..159, WG1 160..303)
      bool ok = true;
      for (int layer = 0; layer < 2 && ok; ++layer) {
        if (!wait_phase_warp(bar_acc, pacc, err)) {
          ok = false;
          break;
        }
        pacc ^= 1;
        fence_after_sync();
        if (wg == 0)
          drain_to_a(tm_row, 0, 160, 300, S.a, r);
        else
          drain_to_a(tm_row, 160, 304, 300, S.a, r);
        fence_proxy_async();
        fence_before_sync();
        mbar_arrive(bar_a);
      }
      if (!ok) break;
      // L3 -> h3 (N = 112: WG0 columns 0..63, WG1 64..111; K columns 100.. = 1, 0, ...)
      if (!wait_phase_warp(bar_acc, pacc, err)) break;
      pacc ^= 1;
      fence_after_sync();
      if (wg == 0)
        drain_to_a(tm_row, 0, 64, 100, S.a, r);
      else
        drain_to_a(tm_row, 64, 112, 100, S.a, r);
      fence_proxy_async();
      fence_before_sync();
      mbar_arrive(bar_a);
      // L4 -> o, conservation layer, BGK + correction + force, store (WG0)
      if (!wait_phase_warp(bar_acc, pacc, err)) break;
      pacc ^= 1;
      fence_after_sync();
      if (wg == 0) {
        uint32_t v0[16], v1[16];
        tmem_ld16(tm_row, v0);
        tmem_ld16(tm_row + 16, v1);
        tmem_wait_ld();
        float o[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) o[i] = __uint_as_float(i < 16 ? v0[i] : v1[i - 16]);
        project(o);
        if (active) {
          const float rw = m.rho * cp.omega;
#pragma unroll
          for (int i = 0; i < Q; ++i) d[i] = fmaf(cp.omega, deq[i] - d[i], d[i]) + rw * o[i];
          const float Fx = cp.fx_y ? __ldg(cp.fx_y + T.y) : 0.f;
          const float Fy = cp.fy_z ? __ldg(cp.fy_z + T.z) : 0.f;
          const float Fz = cp.fz_x ? __ldg(cp.fz_x + x) : 0.f;
          add_edm_force(m, Fx, Fy, Fz, d);
          float *ob = out + (size_t)T.b * Q * vol + ((size_t)T.z * g.ny + T.y) * g.nx + x;
#pragma unroll
          for (int i = 0; i < Q; ++i) ob[(size_t)i * vol] = d[i];
        }
        fence_before_sync();
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = dn[i];
      T = N;
    }
  }

  // ---- teardown: every role has left its loop (normally or on an error)
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (tid == 0 && S.err) atomicOr(timeout_flag, 1);
}

// FP32 packed weights -> BF16 operand tiles in the canonical K-major layout,
// each streamed chunk contiguous, biases in the constant-1 K column.
__global__ void k3_prepare_weights(Mlp3 w, unsigned char *__restrict__ gw) {
  const int total = NH * KX + N4 * K4 + NH * KH + N3 * KH;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    float v = 0.f;
    size_t off;
    if (e < NH * KX) {  // W1: rows n < 300, K 19 inputs, bias at k = 19
      const int n = e / KX, k = e % KX;
      if (n < H1) v = k < Q ? w.w1[n * Q + k] : (k == Q ? w.b1[n] : 0.f);
      off = G_W1 + canon_offset(n, k, KX);
    } else if (e < NH * KX + N4 * K4) {  // W4: rows n < 19, K 100, bias at k = 100
      const int f = e - NH * KX, n = f / K4, k = f % K4;
      if (n < Q) v = k < H3 ? w.w4[n * H3 + k] : (k == H3 ? w.b4[n] : 0.f);
      off = G_W4 + canon_offset(n, k, K4);
    } else if (e < NH * KX + N4 * K4 + NH * KH) {  // W2 chunks
      const int f = e - NH * KX - N4 * K4, n = f / KH, k = f % KH;
      if (n < H2) v = k < H1 ? w.w2[n * H1 + k] : (k == H1 ? w.b2[n] : 0.f);
      const int c = k / KC;
      off = G_W2 + (size_t)c * W2_CHUNK + canon_offset(n, k % KC, chunk_k(c));
    } else {  // W3 chunks
      const int f = e - NH * KX - N4 * K4 - NH * KH, n = f / KH, k = f % KH;
      if (n < H3) v = k < H2 ? w.w3[n * H2 + k] : (k == H2 ? w.b3[n] : 0.f);
      const int c = k / KC;
      off = G_W3 + (size_t)c * W3_CHUNK + canon_offset(n, k % KC, chunk_k(c));
    }
    *reinterpret_cast<__nv_bfloat16 *>(gw + off) = __float2bfloat16_rn(v);
  }
}

}  // namespace

size_t mlp_tc_weight_bytes() { return (size_t)G_BYTES; }

cudaError_t launch_prepare_weights_tc(const Mlp3 &w, void *gw, cudaStream_t s) {
  k3_prepare_weights<<<256, 256, 0, s>>>(w, static_cast<unsigned char *>(gw));
  return cudaGetLastError();
}

cudaError_t launch_step_mlp_tc(const Grid3 &g, const float *in, float *out, const Collide3 &c,
                               const void *gw, int sms, int *flag, int *timeout_flag,
                               cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k3_step_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((g.nx + 127) / 128) * g.ny * g.nz * g.batch;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)(tiles < sms ? tiles : sms);
  if (grid == 0) return cudaSuccess;
  k3_step_mlp_tc<<<grid, THREADS, SMEM_BYTES, s>>>(in, out, g, c,
                                                   static_cast<const unsigned char *>(gw), flag,
                                                   timeout_flag);
  return cudaGetLastError();
}

}  // namespace d3
}  // namespace lbm
