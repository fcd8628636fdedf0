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
// Operands.  The A operands (x and the activations h1, h2, h3, as bf16 pairs)
// live in tensor memory next to the accumulators: the epilogue reads an
// accumulator row with tcgen05.ld and writes the activation row back with
// tcgen05.st, and the next MMA reads A from tensor memory.  That leaves the
// shared memory to the weights: W1, W3 and W4 stay resident (95 KB); W2
// (185 KB, which does not fit beside them) is streamed every tile in K chunks
// of 32 (19,456 bytes) through a 7-slot ring filled by bulk copies
// (cp.async.bulk) from pre-laid-out copies in global memory (the L2 cache
// holds them; CTAs read different replicas to spread the L2 traffic).
//
// Tensor-memory columns: accumulator 0..303, activations (A) 304..455,
// layer-4 output 456..487, x (layer-1 A) 488..503.
//
// Roles in a CTA of 320 threads (one CTA per SM, persistent over a contiguous
// range of tiles):
//   warps 0-3  (WG0)  the epilogue of the low accumulator columns, and the
//                     final update and store of each tile (pull, moments,
//                     conservation layer, BGK, force), done while the next
//                     tile's second GEMM runs;
//   warps 4-7  (WG1)  the epilogue of the high accumulator columns, and the
//                     next tile's layer-1 operand (pull, moments, x), written
//                     while the current tile's third GEMM runs;
//   warp 8            MMA issue (one thread);
//   warp 9            W2 ring producer (one thread).
// Hand-offs are mbarriers: x ready (128 arrivals), A ready (256 arrivals), the
// hidden accumulator ready and the output accumulator ready (MMA commits), and
// the ring's full/empty pairs.  The layer-4 output and x have their own
// tensor-memory columns, so the next tile's first GEMMs run while the output
// is read.  Every wait is bounded; on a time-out the kernel records it in
// shared memory, all roles leave their loops, in-flight copies and MMAs are
// drained with bounded waits, the tensor memory is freed and the timeout flag
// is set.
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
constexpr int KC = 32;     // K per streamed W2 chunk
constexpr int NCHUNK = 10; // 9 chunks of 32 + 1 of 16
constexpr int SLOTS = 7;
constexpr int SLOT_BYTES = NH * KC * 2;  // 19,456
constexpr int W1_BYTES = NH * KX * 2;    // 19,456
constexpr int W4_BYTES = N4 * K4 * 2;    // 7,168
constexpr int W3_BYTES = N3 * KH * 2;    // 68,096
constexpr int W2_CHUNK = NH * KC * 2;    // 19,456 (the last chunk uses half)
// one pre-laid-out copy of the weights in global memory (bytes)
constexpr int G_W1 = 0;
constexpr int G_W4 = G_W1 + W1_BYTES;
constexpr int G_W3 = G_W4 + W4_BYTES;
constexpr int G_W2 = G_W3 + W3_BYTES;
constexpr int G_BYTES = G_W2 + NCHUNK * W2_CHUNK;  // 289,280 per copy
// Every CTA streams the same 185 KB per tile; REPLICAS copies at different
// addresses spread the reads over the L2 cache (CTA b reads copy b % REPLICAS).
constexpr int REPLICAS = 8;

// tensor-memory columns
constexpr uint32_t TM_ACC = 0, TM_A = 304, TM_OUT = 456, TM_X = 488;

constexpr int THREADS = 320;
constexpr int MMA_WARP = 8, PROD_WARP = 9;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct __align__(1024) Smem {
  unsigned char w1[W1_BYTES];
  unsigned char w4[W4_BYTES];
  unsigned char w3[W3_BYTES];
  unsigned char ring[SLOTS][SLOT_BYTES];
  unsigned long long full[SLOTS], empty[SLOTS];
  unsigned long long xready, aready, accready, outready, drain;
  uint32_t taddr;
  int err;
};
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;
static_assert(SMEM_BYTES <= 232448, "shared memory layout too large");

__host__ __device__ constexpr int chunk_k(int c) {
  return c < NCHUNK - 1 ? KC : KH - KC * (NCHUNK - 1);
}

// ---- helpers ------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Non-blocking test of a phase (mbarrier.test_wait never suspends the thread,
// so a completed phase is seen at the next poll).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait that also gives up early once another role has recorded an
// error.  Polls back off with a short sleep so that waiting warps leave the
// issue slots to the warps that work.
template <bool SLEEP = true>
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, volatile int *err) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63u) == 63u && *err) return false;
    if (SLEEP) __nanosleep(20);
  }
  atomicOr(const_cast<int *>(err), 1);
  return false;
}
// The same for a whole warp: every lane waits in mbarrier.try_wait (the
// hardware suspends the warp until the phase completes or a short time limit
// passes) and the lanes agree by a vote, so the warp stays converged for the
// .sync.aligned tensor-memory accesses that follow and waiting warps take no
// issue slots from the MMA and producer warps.  (Lane 0 polling test_wait with
// the other lanes held at a shuffle cost 10 % of the step: 2.46 against
// 2.73 G nodes/s at 256^3.)
__device__ __forceinline__ bool wait_phase_warp(uint32_t bar, uint32_t parity, volatile int *err) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (__any_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    if ((it & 63u) == 63u && __any_sync(0xffffffffu, *err != 0)) return false;
  }
  if ((threadIdx.x & 31) == 0) atomicOr(const_cast<int *>(err), 1);
  return false;
}
// D (+)= A[tmem] * B[smem]^T, one elected thread.
__device__ __forceinline__ void mma_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id,
                                       bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(id), "r"(acc ? 1u : 0u)
      : "memory");
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

// Drain NCOL accumulator columns starting at C0 of this thread's row (loads
// issued before one wait): LeakyReLU, bf16 pairs, into activation columns
// TM_A + C0/2 of the same row.  Columns at or above KVALID are not
// activations: KVALID gets the constant 1 (the bias column), the rest zero.
template <int C0, int NCOL, int KVALID>
__device__ __forceinline__ void drain_cols(uint32_t tm_row) {
  static_assert(NCOL % 16 == 0 && NCOL <= 64, "16..64 columns per drain");
  uint32_t v[NCOL];
#pragma unroll
  for (int q = 0; q < NCOL / 16; ++q)
    tmem_ld16(tm_row + (uint32_t)(TM_ACC + C0 + 16 * q),
              *reinterpret_cast<uint32_t(*)[16]>(v + 16 * q));
  tmem_wait_ld();
  uint32_t p[NCOL / 2];
#pragma unroll
  for (int e = 0; e < NCOL / 2; ++e) {
    const int k = C0 + 2 * e;
    if (k + 1 < KVALID) {
      // LeakyReLU of both values: the two products 0.01 v in one packed
      // multiply (round to nearest per lane, as the scalar form), then max
      const float a0 = __uint_as_float(v[2 * e]), a1 = __uint_as_float(v[2 * e + 1]);
      const float2 s = __fmul2_rn(make_float2(a0, a1), make_float2(LEAKY, LEAKY));
      p[e] = pack2(fmaxf(a0, s.x), fmaxf(a1, s.y));
    } else {
      float h[2];
#pragma unroll
      for (int j = 0; j < 2; ++j)
        h[j] = k + j < KVALID ? lrelu(__uint_as_float(v[2 * e + j]))
                              : (k + j == KVALID ? 1.0f : 0.0f);
      p[e] = pack2(h[0], h[1]);
    }
  }
#pragma unroll
  for (int q = 0; q < NCOL / 32; ++q)
    tmem_st16(tm_row + (uint32_t)(TM_A + C0 / 2 + 16 * q),
              *reinterpret_cast<const uint32_t(*)[16]>(p + 16 * q));
  if (NCOL % 32)
    tmem_st8(tm_row + (uint32_t)(TM_A + C0 / 2 + 16 * (NCOL / 32)),
             *reinterpret_cast<const uint32_t(*)[8]>(p + 16 * (NCOL / 32)));
}

// The low (WG0) or high (WG1) half of a 304-column accumulator -> h (K 0..303).
__device__ __forceinline__ void drain_hidden(int wg, uint32_t tm_row) {
  if (wg == 0) {
    drain_cols<0, 64, H1>(tm_row);
    drain_cols<64, 64, H1>(tm_row);
    drain_cols<128, 32, H1>(tm_row);
  } else {
    drain_cols<160, 64, H1>(tm_row);
    drain_cols<224, 64, H1>(tm_row);
    drain_cols<288, 16, H1>(tm_row);
  }
}

// x = (f - feq)/rho of this thread's node -> its row of the layer-1 operand
// (19 inputs, the constant-1 bias column, zeros) in tensor memory.
__device__ __forceinline__ void write_x(const float d[Q], bool active, uint32_t tm_row) {
  const Moments m = node_moments(d);
  float deq[Q];
  shifted_feq(m, deq);
  const float inv_rho = 1.0f / m.rho;
  float xi[32];
#pragma unroll
  for (int i = 0; i < 32; ++i)
    xi[i] = i < Q ? (active ? (d[i] - deq[i]) * inv_rho : 0.f) : (i == Q ? 1.0f : 0.0f);
  uint32_t p[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) p[e] = pack2(xi[2 * e], xi[2 * e + 1]);
  tmem_st16(tm_row + TM_X, p);
}

// Arrive on `bar` after this thread's tensor-memory stores are complete.
__device__ __forceinline__ void publish(uint32_t bar) {
  tmem_wait_st();
  fence_before_sync();
  mbar_arrive(bar);
}

__global__ void __launch_bounds__(THREADS, 1)
    k3_step_mlp_tc(const float *__restrict__ in, float *__restrict__ out, Grid3 g, Collide3 cp,
                   const unsigned char *__restrict__ gw, int *flag, int *timeout_flag) {
  extern __shared__ unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                      ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *err = &S.err;
  gw += (size_t)(blockIdx.x % REPLICAS) * G_BYTES;

  // ---- prologue: resident weights, barriers, tensor memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(gw + G_W1);
    uint4 *dst = reinterpret_cast<uint4 *>(S.w1);
    for (int e = tid; e < W1_BYTES / 16; e += THREADS) dst[e] = src[e];
    src = reinterpret_cast<const uint4 *>(gw + G_W4);
    dst = reinterpret_cast<uint4 *>(S.w4);
    for (int e = tid; e < W4_BYTES / 16; e += THREADS) dst[e] = src[e];
    src = reinterpret_cast<const uint4 *>(gw + G_W3);
    dst = reinterpret_cast<uint4 *>(S.w3);
    for (int e = tid; e < W3_BYTES / 16; e += THREADS) dst[e] = src[e];
  }
  if (tid == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(smem_u32(&S.full[s]), 1);
      mbar_init(smem_u32(&S.empty[s]), 1);
    }
    mbar_init(smem_u32(&S.xready), 128);
    mbar_init(smem_u32(&S.aready), 256);
    mbar_init(smem_u32(&S.accready), 1);
    mbar_init(smem_u32(&S.outready), 1);
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
  const int ntiles = (int)((long long)tiles_x * g.ny * g.nz * g.batch);
  const int per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
  const int t_begin = blockIdx.x * per + min((int)blockIdx.x, extra);
  const int count = per + ((int)blockIdx.x < extra ? 1 : 0);

  if (warp == PROD_WARP) {
    // ---------------- W2 ring producer
    if (lane == 0) {
      uint32_t used_mask = 0, par_mask = 0;  // per slot: used once; parity of its next use
      int slot = 0;
      bool ok = true;
      for (int t = 0; t < count && ok; ++t) {
        for (int c = 0; c < NCHUNK; ++c) {
          const uint32_t full = smem_u32(&S.full[slot]), empty = smem_u32(&S.empty[slot]);
          const uint32_t bit = 1u << slot;
          // the previous use of this slot must have been consumed
          if ((used_mask & bit) && !wait_phase(empty, (par_mask & bit) ? 0u : 1u, err)) {
            ok = false;
            break;
          }
          const uint32_t bytes = (uint32_t)(NH * chunk_k(c) * 2);
          mbar_arrive_expect_tx(full, bytes);
          bulk_g2s(smem_u32(S.ring[slot]), gw + G_W2 + c * W2_CHUNK, bytes, full);
          used_mask |= bit;
          par_mask ^= bit;
          slot = slot + 1 == SLOTS ? 0 : slot + 1;
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int s = 0; s < SLOTS; ++s)
        if (used_mask & (1u << s)) {
          const uint32_t full = smem_u32(&S.full[s]);
          const uint32_t last = (par_mask & (1u << s)) ? 0u : 1u;  // parity of the last use
          for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
            if (mbar_test(full, last)) break;
        }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue
    if (lane == 0) {
      const uint32_t sw1 = smem_u32(S.w1), sw3 = smem_u32(S.w3), sw4 = smem_u32(S.w4);
      const uint32_t bar_acc = smem_u32(&S.accready), bar_out = smem_u32(&S.outready);
      const uint32_t acc = tmem + TM_ACC, ah = tmem + TM_A, ax = tmem + TM_X;
      constexpr uint32_t ID160 = idesc_bf16_f32(128, 160), ID144 = idesc_bf16_f32(128, 144),
                         ID112 = idesc_bf16_f32(128, 112), ID32 = idesc_bf16_f32(128, 32);
      uint32_t px = 0, pa = 0, par_mask = 0;  // par bit s = parity of the slot's next use
      int slot = 0;
      bool issued = false;
      // the first tile's x (later tiles' x is awaited after the L4 commit)
      bool xok = count > 0 && wait_phase<false>(smem_u32(&S.xready), px, err);
      px ^= 1;
      for (int t = 0; t < count && xok; ++t) {
        // L1: A = x (tensor memory, K 32), B = W1 resident
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < KX / 16; ++s) {
          mma_ta(acc, ax + 8 * s, smem_desc(sw1 + 256 * s, 128, 16 * KX), ID160, s > 0);
          mma_ta(acc + 160, ax + 8 * s, smem_desc(sw1 + 20 * 16 * KX + 256 * s, 128, 16 * KX),
                 ID144, s > 0);
        }
        mma_commit(bar_acc);
        issued = true;
        // L2: A = h1 (tensor memory, K 304), B = streamed W2 chunks, consumed
        // as they land (the stream from the L2 cache sets the pace).  Note that
        // on this GPU the first memory access of a thread after a
        // tcgen05.commit waits until the MMAs it has issued have completed.
        if (!wait_phase<false>(smem_u32(&S.aready), pa, err)) break;
        pa ^= 1;
        fence_after_sync();
        bool ok = true;
        for (int c = 0; c < NCHUNK; ++c) {
          if (!wait_phase<false>(smem_u32(&S.full[slot]), (par_mask >> slot) & 1u, err)) {
            ok = false;
            break;
          }
          par_mask ^= 1u << slot;
          const int kc = chunk_k(c);
          const uint32_t sb = smem_u32(S.ring[slot]);
          for (int s = 0; s < kc / 16; ++s) {
            const uint32_t a = ah + 8 * (2 * c + s);
            const bool accum = c > 0 || s > 0;
            mma_ta(acc, a, smem_desc(sb + 256 * s, 128, 16 * kc), ID160, accum);
            mma_ta(acc + 160, a, smem_desc(sb + 20 * 16 * kc + 256 * s, 128, 16 * kc), ID144,
                   accum);
          }
          mma_commit(smem_u32(&S.empty[slot]));
          slot = slot + 1 == SLOTS ? 0 : slot + 1;
        }
        if (!ok) break;
        mma_commit(bar_acc);
        // L3: A = h2, B = W3 resident (K 304, N 112)
        if (!wait_phase<false>(smem_u32(&S.aready), pa, err)) break;
        pa ^= 1;
        fence_after_sync();
#pragma unroll 1
        for (int s = 0; s < KH / 16; ++s)
          mma_ta(acc, ah + 8 * s, smem_desc(sw3 + 256 * s, 128, 16 * KH), ID112, s > 0);
        mma_commit(bar_acc);
        // L4: A = h3 (K 112), B = W4 resident; its own accumulator columns
        if (!wait_phase<false>(smem_u32(&S.aready), pa, err)) break;
        pa ^= 1;
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < K4 / 16; ++s)
          mma_ta(tmem + TM_OUT, ah + 8 * s, smem_desc(sw4 + 256 * s, 128, 16 * K4), ID32, s > 0);
        mma_commit(bar_out);
        if (t + 1 < count) {  // the next tile's x
          xok = wait_phase<false>(smem_u32(&S.xready), px, err);
          px ^= 1;
        }
      }
      // drain outstanding MMAs before the tensor memory is freed
      if (issued) {
        mma_commit(smem_u32(&S.drain));
        for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
          if (mbar_test(smem_u32(&S.drain), 0)) break;
      }
    }
  } else {
    // ---------------- node and epilogue warpgroups
    const int wg = warp >> 2;
    const int r = tid & 127;
    const uint32_t tm_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t bar_acc = smem_u32(&S.accready), bar_out = smem_u32(&S.outready),
                   bar_a = smem_u32(&S.aready), bar_x = smem_u32(&S.xready);
    uint32_t pacc = 0, pout = 0;
    const size_t vol = g.volume();
    Tile T;
    T.set(t_begin, tiles_x, g.ny, g.nz);
    Tile P = T;  // WG0: the tile whose final update is pending
    float d[Q];  // WG0: populations of tile P; WG1: of the next tile to prepare
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = 0.f;
    if (count > 0 && T.x0 + r < g.nx) pull19(in, g, T, T.x0 + r, d);
    if (wg == 1 && count > 0) {
      write_x(d, T.x0 + r < g.nx, tm_row);
      publish(bar_x);
    }

    // WG0: final update of tile P from the layer-4 output; then load the
    // populations of tile `next` (if any) for its own final update.
    auto finish = [&](const Tile &next, bool have_next) -> bool {
      const int x = P.x0 + r;
      const bool active = x < g.nx;
      const Moments m = node_moments(d);
      {
        const unsigned mask = __ballot_sync(0xffffffffu, active && is_unstable(m));
        if (mask && lane == (__ffs(mask) - 1) && *reinterpret_cast<volatile int *>(flag) == 0)
          atomicOr(flag, 1);
      }
      float deq[Q];
      shifted_feq(m, deq);
      if (!wait_phase_warp(bar_out, pout, err)) return false;
      pout ^= 1;
      fence_after_sync();
      uint32_t v0[16], v1[16];
      tmem_ld16(tm_row + TM_OUT, v0);
      tmem_ld16(tm_row + TM_OUT + 16, v1);
      tmem_wait_ld();
      fence_before_sync();
      float o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) o[i] = __uint_as_float(i < 16 ? v0[i] : v1[i - 16]);
      project(o);
      if (active) {
        const float rw = m.rho * cp.omega;
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = fmaf(cp.omega, deq[i] - d[i], d[i]) + rw * o[i];
        const float Fx = cp.fx_y ? __ldg(cp.fx_y + P.y) : 0.f;
        const float Fy = cp.fy_z ? __ldg(cp.fy_z + P.z) : 0.f;
        const float Fz = cp.fz_x ? __ldg(cp.fz_x + x) : 0.f;
        add_edm_force(m, Fx, Fy, Fz, d);
        float *ob = out + (size_t)P.b * Q * vol + ((size_t)P.z * g.ny + P.y) * g.nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) ob[(size_t)i * vol] = d[i];
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = 0.f;
      if (have_next && next.x0 + r < g.nx) pull19(in, g, next, next.x0 + r, d);
      P = next;
      return true;
    };

    for (int t = 0; t < count; ++t) {
      Tile N = T;
      const bool has_next = t + 1 < count;
      if (has_next) N.set(t_begin + t + 1, tiles_x, g.ny, g.nz);
      // L1 -> h1
      if (!wait_phase_warp(bar_acc, pacc, err)) break;
      pacc ^= 1;
      fence_after_sync();
      drain_hidden(wg, tm_row);
      publish(bar_a);
      if (wg == 0) {
        if (t > 0 && !finish(T, true)) break;  // tile t-1 done; tile t's populations loaded
      } else {
        // the next tile's populations, needed after L2
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = 0.f;
        if (has_next && N.x0 + r < g.nx) pull19(in, g, N, N.x0 + r, d);
      }
      // L2 -> h2
      if (!wait_phase_warp(bar_acc, pacc, err)) break;
      pacc ^= 1;
      fence_after_sync();
      drain_hidden(wg, tm_row);
      publish(bar_a);
      if (wg == 1 && has_next) {
        // the next tile's layer-1 operand (L1 of this tile has read x)
        write_x(d, N.x0 + r < g.nx, tm_row);
        publish(bar_x);
      }
      // L3 -> h3 (K 0..99, the constant column at 100, zeros to 111)
      if (!wait_phase_warp(bar_acc, pacc, err)) break;
      pacc ^= 1;
      fence_after_sync();
      if (wg == 0)
        drain_cols<0, 64, H3>(tm_row);
      else
        drain_cols<64, 48, H3>(tm_row);
      publish(bar_a);
      T = N;
    }
    // WG0: the last tile's final update
    if (wg == 0 && count > 0 && !*err) finish(T, false);
  }

  // ---- teardown: every role has left its loop (normally or on an error)
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (tid == 0 && S.err) atomicOr(timeout_flag, 1);
}

// FP32 packed weights -> BF16 operand tiles in the canonical K-major layout
// (W1, W3, W4 whole; W2 as contiguous K chunks), biases in the constant-1 K
// column, REPLICAS copies.
__global__ void k3_prepare_weights(Mlp3 w, unsigned char *__restrict__ gw) {
  const int total = NH * KX + N4 * K4 + N3 * KH + NH * KH;
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
    } else if (e < NH * KX + N4 * K4 + N3 * KH) {  // W3: rows n < 100, K 300, bias at 300
      const int f = e - NH * KX - N4 * K4, n = f / KH, k = f % KH;
      if (n < H3) v = k < H2 ? w.w3[n * H2 + k] : (k == H2 ? w.b3[n] : 0.f);
      off = G_W3 + canon_offset(n, k, KH);
    } else {  // W2 chunks
      const int f = e - NH * KX - N4 * K4 - N3 * KH, n = f / KH, k = f % KH;
      if (n < H2) v = k < H1 ? w.w2[n * H1 + k] : (k == H1 ? w.b2[n] : 0.f);
      const int c = k / KC;
      off = G_W2 + (size_t)c * W2_CHUNK + canon_offset(n, k % KC, chunk_k(c));
    }
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    for (int rep = 0; rep < REPLICAS; ++rep)
      *reinterpret_cast<__nv_bfloat16 *>(gw + (size_t)rep * G_BYTES + off) = b;
  }
}

}  // namespace

size_t mlp_tc_weight_bytes() { return (size_t)G_BYTES * REPLICAS; }

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
