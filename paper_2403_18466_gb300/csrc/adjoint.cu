// adjoint.cu -- hand-written reverse mode of one unrolled step of the
// learned-collision lattice Boltzmann model (unrolled training, SI section 2),
// FP32 on the CUDA cores, and the deterministic weight-gradient reduction.
//
// Forward step (the one being differentiated): g'(x) = C(f(x)) with the
// pull f_i(x) = g_i(x - c_i) and C the learned collision of Eq. S10-S12 plus
// the EDM force (Eq. S5).  Given lam' = dL/dg', the adjoint step computes
//   lam_i(x - c_i) = [J_C(f(x))^T lam'(x)]_i        (transpose of the pull = push)
//   dtheta        += sum_x (dC/dtheta)^T lam'(x)
// Each CTA owns a fixed list of 128-node tiles (one row segment each),
// recomputes the node's forward values (x, h1, h2, o), runs the chain rule
// backwards per node, scatters lam, and stages the per-node vectors in shared
// memory to accumulate the weight gradient as sums of outer products over the
// tile.  Each CTA writes its own row of partial sums; a second kernel adds
// the rows in a fixed order, so dtheta is bitwise reproducible.
#include "kernels.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int AT = 128;      // threads per CTA = nodes per tile
constexpr int HP = 68;       // padded row stride of the staged hidden vectors
constexpr int XP = 12;       // padded row stride of 9-vectors

struct __align__(16) AdjSmem {
  float w1[HIDDEN][XP];      // [j][k]
  float b1[HIDDEN];
  float w2[HIDDEN][HIDDEN];  // [j][k]
  float w2t[HIDDEN][HIDDEN]; // [k][j]
  float b2[HIDDEN];
  float w3t[HIDDEN][XP];     // [j][i]
  float b3[XP];
  float X[AT][XP];           // x_k, and 1 at k = 9 (bias column)
  float H1[AT][HP];
  float H2[AT][HP];          // h2_j, and 1 at j = 64 (bias column)
  float A1[AT][HP];          // dL/da1
  float A2[AT][HP];          // dL/da2
  float OB[AT][XP];          // dL/do
  float acc[NPARAMS];        // this CTA's running weight gradient
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

// Partial derivatives of feq_i(rho, u) = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2).
__device__ __forceinline__ void feq_partials(float rho, float ux, float uy, int i, float &dr,
                                             float &dux, float &duy) {
  const float cu = (float)cx(i) * ux + (float)cy(i) * uy;
  const float usq = ux * ux + uy * uy;
  dr = wf(i) * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * usq);
  dux = wf(i) * rho * (3.0f * (float)cx(i) + 9.0f * cu * (float)cx(i) - 3.0f * ux);
  duy = wf(i) * rho * (3.0f * (float)cy(i) + 9.0f * cu * (float)cy(i) - 3.0f * uy);
}

__global__ void __launch_bounds__(AT, 1)
    k_adjoint_step(const float *__restrict__ state, const float *__restrict__ lam_next,
                   float *__restrict__ lam_out, int nx, int ny, int batch, CollideParams p,
                   MlpF32 w, float *__restrict__ partials, int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdjSmem &S = *reinterpret_cast<AdjSmem *>(smem_raw);
  const int t = threadIdx.x;
  for (int e = t; e < HIDDEN * XP; e += AT) {
    const int j = e / XP, k = e % XP;
    S.w1[j][k] = k < 9 ? w.w1[j * 9 + k] : 0.f;
    S.w3t[j][k] = k < 9 ? w.w3[k * HIDDEN + j] : 0.f;
  }
  for (int e = t; e < HIDDEN * HIDDEN; e += AT) {
    const int j = e / HIDDEN, k = e % HIDDEN;
    const float v = w.w2[e];
    S.w2[j][k] = v;
    S.w2t[k][j] = v;
  }
  for (int e = t; e < HIDDEN; e += AT) {
    S.b1[e] = w.b1[e];
    S.b2[e] = w.b2[e];
  }
  if (t < XP) S.b3[t] = t < 9 ? w.b3[t] : 0.f;
  for (int e = t; e < NPARAMS; e += AT) S.acc[e] = 0.f;
  __syncthreads();

  const size_t plane = (size_t)nx * ny;
  const int tiles_x = (nx + AT - 1) / AT;
  const long long ntiles = (long long)tiles_x * ny * batch;
  const float omega = p.omega;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = (int)(tile % tiles_x);
    const int y = (int)((tile / tiles_x) % ny);
    const int b = (int)(tile / ((long long)tiles_x * ny));
    const int x = tx * AT + t;
    const bool active = x < nx;
    if (active) {
      const float *gb = state + (size_t)b * Q * plane;
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
      float d[Q], pb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
        const int ys = cy(i) == 0 ? y : (cy(i) == 1 ? ym : yp);
        d[i] = __ldg(gb + i * plane + (size_t)ys * nx + xs);
        pb[i] = __ldg(lam_next + (size_t)b * Q * plane + i * plane + (size_t)y * nx + x);
      }
      // ---- forward recompute ----
      const Moments m = node_moments(d);
      float deq[Q], xin[Q];
      shifted_feq(m, deq);
      const float inv_rho = 1.0f / m.rho;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        xin[i] = (d[i] - deq[i]) * inv_rho;
        S.X[t][i] = xin[i];
      }
      S.X[t][9] = 1.0f;
      for (int j = 0; j < HIDDEN; ++j) {
        float a = S.b1[j];
#pragma unroll
        for (int k = 0; k < 9; ++k) a = fmaf(S.w1[j][k], xin[k], a);
        S.H1[t][j] = tanhf(a);
      }
      float o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) o[i] = S.b3[i];
      for (int j = 0; j < HIDDEN; j += 4) {
        float a0 = S.b2[j], a1 = S.b2[j + 1], a2 = S.b2[j + 2], a3 = S.b2[j + 3];
#pragma unroll 8
        for (int k = 0; k < HIDDEN; ++k) {
          const float h = S.H1[t][k];
          a0 = fmaf(S.w2[j][k], h, a0);
          a1 = fmaf(S.w2[j + 1][k], h, a1);
          a2 = fmaf(S.w2[j + 2][k], h, a2);
          a3 = fmaf(S.w2[j + 3][k], h, a3);
        }
        const float hv[4] = {tanhf(a0), tanhf(a1), tanhf(a2), tanhf(a3)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          S.H2[t][j + q] = hv[q];
#pragma unroll
          for (int i = 0; i < Q; ++i) o[i] = fmaf(S.w3t[j + q][i], hv[q], o[i]);
        }
      }
      S.H2[t][HIDDEN] = 1.0f;
      project9(o);  // o now holds ohat

      // ---- reverse ----
      // post = d + omega (deq - d) + rho omega ohat + fext(rho, u)
      float fb[Q], deqb[Q], ohb[Q];
      float rhob = 0.f, uxb = 0.f, uyb = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fb[i] = pb[i] * (1.0f - omega);
        deqb[i] = pb[i] * omega;
        ohb[i] = m.rho * omega * pb[i];
        rhob = fmaf(omega * pb[i], o[i], rhob);
      }
      const float fx = p.force ? __ldg(p.force + y) : 0.0f;
      if (p.force) {
        // fext = feq(rho, u + a) - feq(rho, u), a = (fx / rho, 0)
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
      project9(ohb);  // dL/do = P^T dL/dohat, P symmetric
#pragma unroll
      for (int i = 0; i < Q; ++i) S.OB[t][i] = ohb[i];
      // dL/da2 = (W3^T dL/do) * (1 - h2^2)
      for (int j = 0; j < HIDDEN; ++j) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) s = fmaf(S.w3t[j][i], ohb[i], s);
        const float h = S.H2[t][j];
        S.A2[t][j] = s * (1.0f - h * h);
      }
      // dL/da1 = (W2^T dL/da2) * (1 - h1^2)
      for (int k = 0; k < HIDDEN; k += 4) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 8
        for (int j = 0; j < HIDDEN; ++j) {
          const float a = S.A2[t][j];
          s0 = fmaf(S.w2t[k][j], a, s0);
          s1 = fmaf(S.w2t[k + 1][j], a, s1);
          s2 = fmaf(S.w2t[k + 2][j], a, s2);
          s3 = fmaf(S.w2t[k + 3][j], a, s3);
        }
        const float sv[4] = {s0, s1, s2, s3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float h = S.H1[t][k + q];
          S.A1[t][k + q] = sv[q] * (1.0f - h * h);
        }
      }
      // dL/dx = W1^T dL/da1
      float xb[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) xb[k] = 0.f;
      for (int j = 0; j < HIDDEN; ++j) {
        const float a = S.A1[t][j];
#pragma unroll
        for (int k = 0; k < Q; ++k) xb[k] = fmaf(S.w1[j][k], a, xb[k]);
      }
      // x = (f - feq) / rho
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fb[i] += xb[i] * inv_rho;
        deqb[i] -= xb[i] * inv_rho;
        rhob -= xb[i] * xin[i] * inv_rho;
      }
      // feq(rho, u)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float dr, dux, duy;
        feq_partials(m.rho, m.ux, m.uy, i, dr, dux, duy);
        rhob = fmaf(deqb[i], dr, rhob);
        uxb = fmaf(deqb[i], dux, uxb);
        uyb = fmaf(deqb[i], duy, uyb);
      }
      // u = j / rho; rho = sum f, j = sum f c
      const float jxb = uxb * inv_rho, jyb = uyb * inv_rho;
      rhob -= (uxb * m.ux + uyb * m.uy) * inv_rho;
      float *lo = lam_out + (size_t)b * Q * plane;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float v = fb[i] + rhob + (float)cx(i) * jxb + (float)cy(i) * jyb;
        const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
        const int ys = cy(i) == 0 ? y : (cy(i) == 1 ? ym : yp);
        lo[i * plane + (size_t)ys * nx + xs] = v;  // lam_i(x - c_i)
      }
    } else {
      // inactive rows of a ragged tile contribute nothing
      for (int k = 0; k < XP; ++k) {
        S.X[t][k] = 0.f;
        S.OB[t][k] = 0.f;
      }
      for (int k = 0; k < HP; ++k) {
        S.H1[t][k] = 0.f;
        S.H2[t][k] = 0.f;
        S.A1[t][k] = 0.f;
        S.A2[t][k] = 0.f;
      }
    }
    __syncthreads();
    // ---- weight gradient: sums of outer products over the tile ----
    {
      // dW2[j][k] += sum_n A2[n][j] H1[n][k]: thread owns a 4 x 8 block
      const int j0 = 4 * (t >> 3), k0 = 8 * (t & 7);
      float c[4][8];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 8; ++q) c[a][q] = 0.f;
      for (int n = 0; n < AT; ++n) {
        const float4 av = *reinterpret_cast<const float4 *>(&S.A2[n][j0]);
        const float4 h0 = *reinterpret_cast<const float4 *>(&S.H1[n][k0]);
        const float4 h1v = *reinterpret_cast<const float4 *>(&S.H1[n][k0 + 4]);
        const float aa[4] = {av.x, av.y, av.z, av.w};
        const float hh[8] = {h0.x, h0.y, h0.z, h0.w, h1v.x, h1v.y, h1v.z, h1v.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 8; ++q) c[a][q] = fmaf(aa[a], hh[q], c[a][q]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 8; ++q) S.acc[OFF_W2 + (j0 + a) * HIDDEN + k0 + q] += c[a][q];
    }
    {
      // [dW1 | db1][j][k] += sum_n A1[n][j] [x | 1][n][k]: 64 x 10 entries, 5 per thread
      const int j = t >> 1, kb = 5 * (t & 1);
      float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int n = 0; n < AT; ++n) {
        const float a = S.A1[n][j];
#pragma unroll
        for (int q = 0; q < 5; ++q) c[q] = fmaf(a, S.X[n][kb + q], c[q]);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int k = kb + q;
        if (k < 9) S.acc[OFF_W1 + j * 9 + k] += c[q];
        else S.acc[OFF_B1 + j] += c[q];
      }
    }
    {
      // [dW3 | db3][i][j] += sum_n OB[n][i] [h2 | 1][n][j]: 9 x 65 entries
      for (int e = t; e < 9 * (HIDDEN + 1); e += AT) {
        const int i = e / (HIDDEN + 1), j = e % (HIDDEN + 1);
        float c = 0.f;
        for (int n = 0; n < AT; ++n) c = fmaf(S.OB[n][i], S.H2[n][j], c);
        if (j < HIDDEN) S.acc[OFF_W3 + i * HIDDEN + j] += c;
        else S.acc[OFF_B3 + i] += c;
      }
      // db2[j] += sum_n A2[n][j]
      if (t < HIDDEN) {
        float c = 0.f;
        for (int n = 0; n < AT; ++n) c += S.A2[n][t];
        S.acc[OFF_B2 + t] += c;
      }
    }
    __syncthreads();
  }
  float *row = partials + (size_t)blockIdx.x * NPARAMS;
  for (int e = t; e < NPARAMS; e += AT) row[e] = accumulate ? row[e] + S.acc[e] : S.acc[e];
}

// dW[e] = sum over rows r (in order) of partials[r][e], FP64 accumulation.
__global__ void k_reduce_dw(const float *__restrict__ partials, int rows, float *__restrict__ dW) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPARAMS) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += (double)partials[(size_t)r * NPARAMS + e];
  dW[e] = (float)s;
}

}  // namespace

int adjoint_blocks(const Grid &g, int sms) {
  const long long tiles = (long long)((g.nx + AT - 1) / AT) * g.ny * g.batch;
  return (int)(tiles < sms ? tiles : sms);
}

size_t adjoint_smem_bytes() { return sizeof(AdjSmem); }

cudaError_t launch_adjoint_step(const Grid &g, const float *state_n, const float *lam_next,
                                float *lam_out, const CollideParams &p, const MlpF32 &w,
                                float *dw_partials, int rows, int accumulate, cudaStream_t s) {
  static bool attr_set = false;  // per-process; the attribute is per function
  const size_t smem = sizeof(AdjSmem);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_step,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_adjoint_step<<<rows, AT, smem, s>>>(state_n, lam_next, lam_out, g.nx, g.ny, g.batch, p, w,
                                        dw_partials, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_reduce_dw(const float *dw_partials, int rows, float *dW, cudaStream_t s) {
  k_reduce_dw<<<(NPARAMS + 255) / 256, 256, 0, s>>>(dw_partials, rows, dW);
  return cudaGetLastError();
}

}  // namespace lbm
