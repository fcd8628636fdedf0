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
// tile.  The staging buffers hold one CTA per SM, so the per-node phase keeps
// its vectors in registers (up to 255 per thread are free at 128 threads) and
// reads the weights as float4 broadcasts.  Each CTA writes its own row of partial sums; a second kernel adds
// the rows in a fixed order, so dtheta is bitwise reproducible.
#include "kernels.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int AT = 128;      // threads per CTA = nodes per tile
constexpr int HP = 68;       // padded row stride of the staged hidden vectors
constexpr int XP = 12;       // padded row stride of 9-vectors
// hidden units per group of independent accumulators in the 64 x 64 products
// (8 or 16 measured slower)
constexpr int G2 = 4;
static_assert(G2 % 4 == 0 && HIDDEN % G2 == 0, "accumulator groups");

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
      for (int i = 0; i < Q; ++i) xin[i] = (d[i] - deq[i]) * inv_rho;
      // Per-node vectors are written to (and read from) this thread's rows of
      // the staging buffers with 16-byte accesses (a row stride of 68 floats
      // keeps those free of bank conflicts); weights are read as float4
      // broadcasts.
      {
        float4 *xr = reinterpret_cast<float4 *>(&S.X[t][0]);
        xr[0] = make_float4(xin[0], xin[1], xin[2], xin[3]);
        xr[1] = make_float4(xin[4], xin[5], xin[6], xin[7]);
        xr[2] = make_float4(xin[8], 1.0f, 0.f, 0.f);
      }
      float h1[HIDDEN];
#pragma unroll
      for (int j = 0; j < HIDDEN; ++j) {
        const float4 wa = *reinterpret_cast<const float4 *>(&S.w1[j][0]);
        const float4 wb = *reinterpret_cast<const float4 *>(&S.w1[j][4]);
        float a = S.b1[j];
        a = fmaf(wa.x, xin[0], a);
        a = fmaf(wa.y, xin[1], a);
        a = fmaf(wa.z, xin[2], a);
        a = fmaf(wa.w, xin[3], a);
        a = fmaf(wb.x, xin[4], a);
        a = fmaf(wb.y, xin[5], a);
        a = fmaf(wb.z, xin[6], a);
        a = fmaf(wb.w, xin[7], a);
        a = fmaf(S.w1[j][8], xin[8], a);
        h1[j] = tanhf(a);
      }
      {
        float4 *hr = reinterpret_cast<float4 *>(&S.H1[t][0]);
#pragma unroll
        for (int q = 0; q < HIDDEN / 4; ++q)
          hr[q] = make_float4(h1[4 * q], h1[4 * q + 1], h1[4 * q + 2], h1[4 * q + 3]);
      }
      float o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) o[i] = S.b3[i];
      for (int j = 0; j < HIDDEN; j += G2) {
        float acc[G2];
        const float4 *rw[G2];
#pragma unroll
        for (int g = 0; g < G2; ++g) {
          acc[g] = S.b2[j + g];
          rw[g] = reinterpret_cast<const float4 *>(&S.w2[j + g][0]);
        }
#pragma unroll
        for (int k4 = 0; k4 < HIDDEN / 4; ++k4) {
          float4 u[G2];
#pragma unroll
          for (int g = 0; g < G2; ++g) u[g] = rw[g][k4];
          const float *h = &h1[4 * k4];
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].x, h[0], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].y, h[1], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].z, h[2], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].w, h[3], acc[g]);
        }
        float hv[G2];
#pragma unroll
        for (int g = 0; g < G2; ++g) hv[g] = tanhf(acc[g]);
#pragma unroll
        for (int g = 0; g < G2; g += 4)
          *reinterpret_cast<float4 *>(&S.H2[t][j + g]) =
              make_float4(hv[g], hv[g + 1], hv[g + 2], hv[g + 3]);
#pragma unroll
        for (int q = 0; q < G2; ++q) {
          const float4 c0 = *reinterpret_cast<const float4 *>(&S.w3t[j + q][0]);
          const float4 c1 = *reinterpret_cast<const float4 *>(&S.w3t[j + q][4]);
          o[0] = fmaf(c0.x, hv[q], o[0]);
          o[1] = fmaf(c0.y, hv[q], o[1]);
          o[2] = fmaf(c0.z, hv[q], o[2]);
          o[3] = fmaf(c0.w, hv[q], o[3]);
          o[4] = fmaf(c1.x, hv[q], o[4]);
          o[5] = fmaf(c1.y, hv[q], o[5]);
          o[6] = fmaf(c1.z, hv[q], o[6]);
          o[7] = fmaf(c1.w, hv[q], o[7]);
          o[8] = fmaf(S.w3t[j + q][8], hv[q], o[8]);
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
      {
        float4 *orow = reinterpret_cast<float4 *>(&S.OB[t][0]);
        orow[0] = make_float4(ohb[0], ohb[1], ohb[2], ohb[3]);
        orow[1] = make_float4(ohb[4], ohb[5], ohb[6], ohb[7]);
        orow[2] = make_float4(ohb[8], 0.f, 0.f, 0.f);
      }
      // dL/da2 = (W3^T dL/do) * (1 - h2^2), kept in registers
      float a2v[HIDDEN];
#pragma unroll
      for (int j4 = 0; j4 < HIDDEN / 4; ++j4) {
        const float4 h4 = *reinterpret_cast<const float4 *>(&S.H2[t][4 * j4]);
        const float hh[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * j4 + q;
          const float4 c0 = *reinterpret_cast<const float4 *>(&S.w3t[j][0]);
          const float4 c1 = *reinterpret_cast<const float4 *>(&S.w3t[j][4]);
          float s = 0.f;
          s = fmaf(c0.x, ohb[0], s);
          s = fmaf(c0.y, ohb[1], s);
          s = fmaf(c0.z, ohb[2], s);
          s = fmaf(c0.w, ohb[3], s);
          s = fmaf(c1.x, ohb[4], s);
          s = fmaf(c1.y, ohb[5], s);
          s = fmaf(c1.z, ohb[6], s);
          s = fmaf(c1.w, ohb[7], s);
          s = fmaf(S.w3t[j][8], ohb[8], s);
          const float h = hh[q];
          a2v[j] = s * (1.0f - h * h);
        }
        *reinterpret_cast<float4 *>(&S.A2[t][4 * j4]) =
            make_float4(a2v[4 * j4], a2v[4 * j4 + 1], a2v[4 * j4 + 2], a2v[4 * j4 + 3]);
      }
      // dL/da1 = (W2^T dL/da2) * (1 - h1^2), and dL/dx = W1^T dL/da1
      float xb[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) xb[k] = 0.f;
      for (int k = 0; k < HIDDEN; k += G2) {
        float acc[G2];
        const float4 *rw[G2];
#pragma unroll
        for (int g = 0; g < G2; ++g) {
          acc[g] = 0.f;
          rw[g] = reinterpret_cast<const float4 *>(&S.w2t[k + g][0]);
        }
#pragma unroll
        for (int j4 = 0; j4 < HIDDEN / 4; ++j4) {
          float4 u[G2];
#pragma unroll
          for (int g = 0; g < G2; ++g) u[g] = rw[g][j4];
          const float *a = &a2v[4 * j4];
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].x, a[0], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].y, a[1], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].z, a[2], acc[g]);
#pragma unroll
          for (int g = 0; g < G2; ++g) acc[g] = fmaf(u[g].w, a[3], acc[g]);
        }
        float av[G2];
#pragma unroll
        for (int g = 0; g < G2; g += 4) {
          const float4 h4 = *reinterpret_cast<const float4 *>(&S.H1[t][k + g]);
          const float hh[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float h = hh[q];
            av[g + q] = acc[g + q] * (1.0f - h * h);
          }
          *reinterpret_cast<float4 *>(&S.A1[t][k + g]) =
              make_float4(av[g], av[g + 1], av[g + 2], av[g + 3]);
        }
#pragma unroll
        for (int q = 0; q < G2; ++q) {
          const float4 wa = *reinterpret_cast<const float4 *>(&S.w1[k + q][0]);
          const float4 wb = *reinterpret_cast<const float4 *>(&S.w1[k + q][4]);
          xb[0] = fmaf(wa.x, av[q], xb[0]);
          xb[1] = fmaf(wa.y, av[q], xb[1]);
          xb[2] = fmaf(wa.z, av[q], xb[2]);
          xb[3] = fmaf(wa.w, av[q], xb[3]);
          xb[4] = fmaf(wb.x, av[q], xb[4]);
          xb[5] = fmaf(wb.y, av[q], xb[5]);
          xb[6] = fmaf(wb.z, av[q], xb[6]);
          xb[7] = fmaf(wb.w, av[q], xb[7]);
          xb[8] = fmaf(S.w1[k + q][8], av[q], xb[8]);
        }
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
      // [dW3 | db3][i][j] += sum_n OB[n][i] [h2 | 1][n][j]: 9 x 65 entries,
      // thread j < 65 owning column j (dL/do rows read as float4 broadcasts)
      if (t <= HIDDEN) {
        const int j = t;
        float c[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) c[i] = 0.f;
        for (int n = 0; n < AT; ++n) {
          const float4 o0 = *reinterpret_cast<const float4 *>(&S.OB[n][0]);
          const float4 o1 = *reinterpret_cast<const float4 *>(&S.OB[n][4]);
          const float o8 = S.OB[n][8];
          const float h = S.H2[n][j];
          c[0] = fmaf(o0.x, h, c[0]);
          c[1] = fmaf(o0.y, h, c[1]);
          c[2] = fmaf(o0.z, h, c[2]);
          c[3] = fmaf(o0.w, h, c[3]);
          c[4] = fmaf(o1.x, h, c[4]);
          c[5] = fmaf(o1.y, h, c[5]);
          c[6] = fmaf(o1.z, h, c[6]);
          c[7] = fmaf(o1.w, h, c[7]);
          c[8] = fmaf(o8, h, c[8]);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (j < HIDDEN) S.acc[OFF_W3 + i * HIDDEN + j] += c[i];
          else S.acc[OFF_B3 + i] += c[i];
        }
      } else {
        // db2[j] += sum_n A2[n][j] on the remaining threads
        for (int j = t - (HIDDEN + 1); j < HIDDEN; j += AT - (HIDDEN + 1)) {
          float c = 0.f;
          for (int n = 0; n < AT; ++n) c += S.A2[n][j];
          S.acc[OFF_B2 + j] += c;
        }
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
