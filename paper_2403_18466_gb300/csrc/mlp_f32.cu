// mlp_f32.cu -- fused pull-stream + learned collision, all in FP32 on the
// CUDA cores (the correctness companion of the tensor-core kernel).
//
// Per node (Eq. S10-S12 with the network of this library):
//   x     = (f - feq) / rho                     (9, intensive input)
//   h1    = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3
//   ohat  = o - mean(o) - c_x (sum o c_x)/6 - c_y (sum o c_y)/6   (Eqs. S11-S12, D2Q9)
//   f'    = f + (feq - f)/tau + (rho/tau) ohat + f_ext            (Eq. S10, Eq. S5)
// One thread per node; the weights live in shared memory (21.5 KB) and are
// read as warp-wide broadcasts.  About 5.3 k FMAs and 128 tanh per node, so
// the kernel is bound by the FP32 pipe, not by HBM.
#include "kernels.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int THREADS = 128;
constexpr int ROWS_PER_BLOCK = 8;
// Layer 2 computes G2 hidden units at a time (independent accumulator
// chains), and the kernel is held to 128 registers so that four CTAs share
// an SM: 3.0 against 2.9 G nodes/s for one unit at a time and 140 registers
// (2048^2); four units at a time, or more registers, measured slower.
constexpr int G2 = 2;
constexpr int MIN_BLOCKS = 4;

struct __align__(16) SmemWeights {
  float w1[HIDDEN][12];  // [j][k], k < 9 used, padded to 3 float4
  float b1[HIDDEN];
  float w2[HIDDEN][HIDDEN];
  float b2[HIDDEN];
  float w3t[HIDDEN][12];  // transposed: [j][i], i < 9 used
  float b3[12];
};

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

__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
    k_step_mlp_f32(const float *__restrict__ in, float *__restrict__ out, int nx, int ny,
                   CollideParams p, MlpF32 w, int *flag) {
  __shared__ SmemWeights sw;
  for (int t = threadIdx.x; t < HIDDEN * 12; t += THREADS) {
    const int j = t / 12, k = t % 12;
    sw.w1[j][k] = k < 9 ? w.w1[j * 9 + k] : 0.f;
    sw.w3t[j][k] = k < 9 ? w.w3[k * HIDDEN + j] : 0.f;
  }
  for (int t = threadIdx.x; t < HIDDEN * HIDDEN; t += THREADS) sw.w2[t / HIDDEN][t % HIDDEN] = w.w2[t];
  for (int t = threadIdx.x; t < HIDDEN; t += THREADS) {
    sw.b1[t] = w.b1[t];
    sw.b2[t] = w.b2[t];
  }
  if (threadIdx.x < 12) sw.b3[threadIdx.x] = threadIdx.x < 9 ? w.b3[threadIdx.x] : 0.f;
  __syncthreads();

  const int x = blockIdx.x * THREADS + threadIdx.x;
  if (x >= nx) return;
  const size_t plane = (size_t)nx * ny;
  const float *gb = in + (size_t)blockIdx.z * Q * plane;
  float *ob = out + (size_t)blockIdx.z * Q * plane;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;

  for (int r = 0; r < ROWS_PER_BLOCK; ++r) {
    const int y = blockIdx.y * ROWS_PER_BLOCK + r;
    if (y >= ny) break;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
      const int ys = cy(i) == 0 ? y : (cy(i) == 1 ? ym : yp);
      d[i] = __ldg(gb + i * plane + (size_t)ys * nx + xs);
    }
    const Moments m = node_moments(d);
    flag_unstable(is_unstable(m), flag);
    float deq[Q], xin[Q];
    shifted_feq(m, deq);
    const float inv_rho = 1.0f / m.rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * inv_rho;

    float h1[HIDDEN];
#pragma unroll
    for (int j = 0; j < HIDDEN; ++j) {
      const float4 a = *reinterpret_cast<const float4 *>(&sw.w1[j][0]);
      const float4 b = *reinterpret_cast<const float4 *>(&sw.w1[j][4]);
      float acc = sw.b1[j];
      acc = fmaf(a.x, xin[0], acc); acc = fmaf(a.y, xin[1], acc);
      acc = fmaf(a.z, xin[2], acc); acc = fmaf(a.w, xin[3], acc);
      acc = fmaf(b.x, xin[4], acc); acc = fmaf(b.y, xin[5], acc);
      acc = fmaf(b.z, xin[6], acc); acc = fmaf(b.w, xin[7], acc);
      acc = fmaf(sw.w1[j][8], xin[8], acc);
      h1[j] = tanhf(acc);
    }
    float o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) o[i] = sw.b3[i];
    for (int j = 0; j < HIDDEN; j += G2) {
      float acc[G2];
      const float4 *wr[G2];
#pragma unroll
      for (int g = 0; g < G2; ++g) {
        acc[g] = sw.b2[j + g];
        wr[g] = reinterpret_cast<const float4 *>(&sw.w2[j + g][0]);
      }
#pragma unroll
      for (int k4 = 0; k4 < HIDDEN / 4; ++k4) {
        float4 a[G2];
#pragma unroll
        for (int g = 0; g < G2; ++g) a[g] = wr[g][k4];
#pragma unroll
        for (int g = 0; g < G2; ++g) {
          acc[g] = fmaf(a[g].x, h1[4 * k4 + 0], acc[g]);
          acc[g] = fmaf(a[g].y, h1[4 * k4 + 1], acc[g]);
          acc[g] = fmaf(a[g].z, h1[4 * k4 + 2], acc[g]);
          acc[g] = fmaf(a[g].w, h1[4 * k4 + 3], acc[g]);
        }
      }
#pragma unroll
      for (int g = 0; g < G2; ++g) {
        const float h2 = tanhf(acc[g]);
        const float4 c0 = *reinterpret_cast<const float4 *>(&sw.w3t[j + g][0]);
        const float4 c1 = *reinterpret_cast<const float4 *>(&sw.w3t[j + g][4]);
        o[0] = fmaf(c0.x, h2, o[0]); o[1] = fmaf(c0.y, h2, o[1]);
        o[2] = fmaf(c0.z, h2, o[2]); o[3] = fmaf(c0.w, h2, o[3]);
        o[4] = fmaf(c1.x, h2, o[4]); o[5] = fmaf(c1.y, h2, o[5]);
        o[6] = fmaf(c1.z, h2, o[6]); o[7] = fmaf(c1.w, h2, o[7]);
        o[8] = fmaf(sw.w3t[j + g][8], h2, o[8]);
      }
    }
    project9(o);
    const float rw = m.rho * p.omega;  // rho / tau
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = fmaf(p.omega, deq[i] - d[i], d[i]) + rw * o[i];
    add_edm_force_x(m, p.force ? __ldg(p.force + y) : 0.0f, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) ob[i * plane + (size_t)y * nx + x] = d[i];
  }
}

}  // namespace

cudaError_t launch_step_mlp_f32(const Grid &g, const float *in, float *out,
                                const CollideParams &p, const MlpF32 &w, int *flag,
                                cudaStream_t s) {
  dim3 grid((g.nx + THREADS - 1) / THREADS, (g.ny + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK, g.batch);
  k_step_mlp_f32<<<grid, THREADS, 0, s>>>(in, out, g.nx, g.ny, p, w, flag);
  return cudaGetLastError();
}

}  // namespace lbm
