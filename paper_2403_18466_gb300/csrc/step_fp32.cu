// step_fp32.cu -- HBM-bound FP32 kernels: the fused pull-stream + BGK /
// Smagorinsky-BGK step (+ EDM forcing), and the data-movement kernels
// around it (state in/out, equilibrium init, moments, box and subsampling
// filters, full-field and node-subset losses, push/pull of a field).
//
// Step kernel (Eq. S2 with the stream/collide split of the Methods section):
// each node pulls f_i(x) = g_i(x - c_i) from the previous buffer, collides
// (Eq. S3, or SI section 1 for Smagorinsky), adds the EDM force (Eq. S5) and
// stores into the next buffer at x.  Algorithmic traffic: 36 B read + 36 B
// written per node (FP32 D2Q9).
//
// Fast path (nx % 4 == 0): one thread owns 4 consecutive nodes of a row.
// Every plane row is read with aligned 128-bit loads; the one value that a
// shifted plane (c_x = +-1) needs from the neighbouring 4-node group comes
// from the adjacent lane by a warp shuffle, and only the warp's edge lanes
// (and the periodic wrap) issue an extra scalar load.  Stores are aligned
// 128-bit.  Other widths take a one-node-per-thread kernel.
#include "approx.cuh"
#include "kernels.h"
#include "lattice.cuh"
#include "umma.cuh"

namespace lbm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int VEC_THREADS = 128;  // 512 nodes of one row per block
constexpr int SCALAR_THREADS = 128;

enum { KIND_BGK = 0, KIND_SMAG = 1 };

// Collide one node in place (shifted representation), add the force.
// Returns true if the node is unstable (|u| >= 0.4 or not finite).
template <int KIND>
__device__ __forceinline__ bool collide_node(float d[Q], const CollideParams &p, float fx) {
  const Moments m = node_moments(d);
  const bool bad = is_unstable(m);
  float deq[Q];
  shifted_feq(m, deq);
  float omega = p.omega;
  if (KIND == KIND_SMAG) {
    // Pi^neq_ab = sum_i c_ia c_ib (f_i - feq_i); tau_eff closed form (SI sec. 1)
    float n[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = d[i] - deq[i];
    const float pxx = (n[1] + n[3]) + ((n[5] + n[6]) + (n[7] + n[8]));
    const float pyy = (n[2] + n[4]) + ((n[5] + n[6]) + (n[7] + n[8]));
    const float pxy = (n[5] - n[6]) + (n[7] - n[8]);
    omega = smagorinsky_omega(pxx * pxx + 2.0f * pxy * pxy + pyy * pyy, m.inv_rho, p.tau,
                              p.tau0_sq, p.smag_c18);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = bgk_relax(d[i], deq[i], omega);
  add_edm_force_x(m, fx, d);  // fx = 0 without forcing
  return bad;
}

__device__ __forceinline__ float4 ldg4(const float *p) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}

// Values g(x0 - CXI .. x0 + 3 - CXI) of one plane row, for the 4-node group
// starting at x0 (x0 % 4 == 0).  All lanes must call it (warp shuffles).
template <int CXI>
__device__ __forceinline__ void pull4(const float *__restrict__ row, int x0, int nx, int lane,
                                      bool active, float v[4]) {
  const float4 a = active ? ldg4(row + x0) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (CXI == 0) {
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if (CXI == 1) {  // needs x0 - 1 .. x0 + 2
    float prev = __shfl_up_sync(FULL, a.w, 1);
    if (active && lane == 0) prev = __ldg(row + (x0 == 0 ? nx - 1 : x0 - 1));
    v[0] = prev; v[1] = a.x; v[2] = a.y; v[3] = a.z;
  } else {  // CXI == -1: needs x0 + 1 .. x0 + 4
    float next = __shfl_down_sync(FULL, a.x, 1);
    if (active && (lane == 31 || x0 + 4 >= nx)) next = __ldg(row + (x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4));
    v[0] = a.y; v[1] = a.z; v[2] = a.w; v[3] = next;
  }
}

template <int I>
__device__ __forceinline__ void pull_plane4(const float *__restrict__ gb, size_t plane, int nx,
                                            int y, int ym, int yp, int x0, int lane, bool active,
                                            float v[Q][4]) {
  const int ys = cy(I) == 0 ? y : (cy(I) == 1 ? ym : yp);  // source row y - c_iy
  pull4<cx(I)>(gb + I * plane + (size_t)ys * nx, x0, nx, lane, active, v[I]);
}

template <int KIND>
__global__ void __launch_bounds__(VEC_THREADS)
    k_step_vec(const float *__restrict__ in, float *__restrict__ out, int nx, int ny,
               CollideParams p, int *flag) {
  umma::griddep_wait();  // launched as a dependent of the previous step
  umma::griddep_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int x0 = (blockIdx.x * VEC_THREADS + threadIdx.x) * 4;
  const int y = blockIdx.y;
  const size_t plane = (size_t)nx * ny;
  const float *gb = in + (size_t)blockIdx.z * Q * plane;
  float *ob = out + (size_t)blockIdx.z * Q * plane;
  const bool active = x0 < nx;
  const int ym = y == 0 ? ny - 1 : y - 1;
  const int yp = y == ny - 1 ? 0 : y + 1;
  float v[Q][4];
  pull_plane4<0>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<1>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<2>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<3>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<4>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<5>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<6>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<7>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  pull_plane4<8>(gb, plane, nx, y, ym, yp, x0, lane, active, v);
  const float fx = p.force ? __ldg(p.force + y) : 0.0f;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = v[i][k];
    bad |= collide_node<KIND>(d, p, fx);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i][k] = d[i];
  }
  flag_unstable(bad && active, flag);
  if (!active) return;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    *reinterpret_cast<float4 *>(ob + i * plane + (size_t)y * nx + x0) =
        make_float4(v[i][0], v[i][1], v[i][2], v[i][3]);
}

// Gather the 9 pulled values of node (x, y): d_i = g_i(x - c_i).
__device__ __forceinline__ void pull_node(const float *__restrict__ gb, size_t plane, int nx,
                                          int ny, int x, int y, float d[Q]) {
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = cx(i) == 0 ? x : (cx(i) == 1 ? xm : xp);
    const int ys = cy(i) == 0 ? y : (cy(i) == 1 ? ym : yp);
    d[i] = __ldg(gb + i * plane + (size_t)ys * nx + xs);
  }
}

template <int KIND>
__global__ void __launch_bounds__(SCALAR_THREADS)
    k_step_scalar(const float *__restrict__ in, float *__restrict__ out, int nx, int ny,
                  CollideParams p, int *flag) {
  umma::griddep_wait();  // launched as a dependent of the previous step
  umma::griddep_launch_dependents();
  const int x = blockIdx.x * SCALAR_THREADS + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const size_t plane = (size_t)nx * ny;
  const float *gb = in + (size_t)blockIdx.z * Q * plane;
  float *ob = out + (size_t)blockIdx.z * Q * plane;
  float d[Q];
  pull_node(gb, plane, nx, ny, x, y, d);
  const bool bad = collide_node<KIND>(d, p, p.force ? __ldg(p.force + y) : 0.0f);
  flag_unstable(bad, flag);
#pragma unroll
  for (int i = 0; i < Q; ++i) ob[i * plane + (size_t)y * nx + x] = d[i];
}

// Programmatic dependent launch: the kernel waits for the previous kernel on
// the stream before its first global access, so its CTAs may be scheduled
// while that kernel's last CTAs finish (it hides the launch gap between steps).
template <int KIND>
cudaError_t launch_step(const Grid &g, const float *in, float *out, const CollideParams &p,
                        int *flag, cudaStream_t s) {
  const bool vec = g.nx % 4 == 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = vec ? dim3((g.nx / 4 + VEC_THREADS - 1) / VEC_THREADS, g.ny, g.batch)
                    : dim3((g.nx + SCALAR_THREADS - 1) / SCALAR_THREADS, g.ny, g.batch);
  cfg.blockDim = dim3(vec ? VEC_THREADS : SCALAR_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (vec) return cudaLaunchKernelEx(&cfg, k_step_vec<KIND>, in, out, g.nx, g.ny, p, flag);
  return cudaLaunchKernelEx(&cfg, k_step_scalar<KIND>, in, out, g.nx, g.ny, p, flag);
}

// ---------------------------------------------------------------------------
// Node-parallel helpers: one thread per node, grid (ceil(nx/128), ny, batch).
// ---------------------------------------------------------------------------
constexpr int NT = 128;

__device__ __forceinline__ bool node_index(int nx, int &x, int &y, int &b) {
  x = blockIdx.x * NT + threadIdx.x;
  y = blockIdx.y;
  b = blockIdx.z;
  return x < nx;
}

dim3 node_grid(const Grid &g) { return dim3((g.nx + NT - 1) / NT, g.ny, g.batch); }

// state_i(x) = f_i(x + c_i) - w_i  (anti-streaming, SI section 2 step 4)
__global__ void k_set_state(const float *__restrict__ f, float *__restrict__ st, int nx, int ny) {
  int x, y, b;
  if (!node_index(nx, x, y, b)) return;
  const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrap_index(x + cx(i), nx), ys = wrap_index(y + cy(i), ny);
    st[base + i * plane + (size_t)y * nx + x] = f[base + i * plane + (size_t)ys * nx + xs] - wf(i);
  }
}

// f_i(x) = state_i(x - c_i) + w_i
__global__ void k_get_state(const float *__restrict__ st, float *__restrict__ f, int nx, int ny) {
  int x, y, b;
  if (!node_index(nx, x, y, b)) return;
  const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
  float d[Q];
  pull_node(st + base, plane, nx, ny, x, y, d);
#pragma unroll
  for (int i = 0; i < Q; ++i) f[base + i * plane + (size_t)y * nx + x] = d[i] + wf(i);
}

// feq(rho, u) at node x becomes the pre-collision state: written to x - c_i.
__global__ void k_init_equilibrium(const float *__restrict__ rho, const float *__restrict__ ux,
                                   const float *__restrict__ uy, float *__restrict__ st, int nx,
                                   int ny) {
  int x, y, b;
  if (!node_index(nx, x, y, b)) return;
  const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
  const size_t n = (size_t)b * plane + (size_t)y * nx + x;
  Moments m;
  m.rho = rho[n];
  m.drho = m.rho - 1.0f;
  m.ux = ux[n];
  m.uy = uy[n];
  float deq[Q];
  shifted_feq(m, deq);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrap_index(x - cx(i), nx), ys = wrap_index(y - cy(i), ny);
    st[base + i * plane + (size_t)ys * nx + xs] = deq[i];
  }
}

__global__ void k_moments(const float *__restrict__ st, float *rho, float *ux, float *uy, int nx,
                          int ny) {
  int x, y, b;
  if (!node_index(nx, x, y, b)) return;
  const size_t plane = (size_t)nx * ny;
  float d[Q];
  pull_node(st + (size_t)b * Q * plane, plane, nx, ny, x, y, d);
  const Moments m = node_moments(d);
  const size_t n = (size_t)b * plane + (size_t)y * nx + x;
  if (rho) rho[n] = m.rho;
  if (ux) ux[n] = m.ux;
  if (uy) uy[n] = m.uy;
}

// f_coarse_i(I, J) = w_i + mean over the cg x cg block of d_i(x - c_i).
// One thread per coarse node; FP64 accumulation of the block sum.
__global__ void k_box_filter(const float *__restrict__ st, float *__restrict__ fc, int nx, int ny,
                             int cg) {
  const int NX = nx / cg, NY = ny / cg;
  const int I = blockIdx.x * NT + threadIdx.x, J = blockIdx.y, b = blockIdx.z;
  if (I >= NX) return;
  const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
  const size_t cplane = (size_t)NX * NY;
  const double inv = 1.0 / ((double)cg * cg);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double s = 0.0;
    for (int a = 0; a < cg; ++a) {
      const int ys = wrap_index(J * cg + a - cy(i), ny);
      const float *row = st + base + i * plane + (size_t)ys * nx;
      for (int c = 0; c < cg; ++c) s += (double)__ldg(row + wrap_index(I * cg + c - cx(i), nx));
    }
    fc[(size_t)b * Q * cplane + i * cplane + (size_t)J * NX + I] = (float)(s * inv) + wf(i);
  }
}

// Velocity loss: per-node squared error, block partial sums (fixed order),
// and optionally dL/df_i = s ((u - u_t).(c_i - u)) / rho, s = 1/(N B).
__global__ void k_velocity_loss(const float *__restrict__ st, const float *__restrict__ utx,
                                const float *__restrict__ uty, float *__restrict__ partials,
                                float *__restrict__ dL_df, int nx, int ny, float s) {
  __shared__ float red[NT];
  int x, y, b;
  const bool ok = node_index(nx, x, y, b);
  float e = 0.0f;
  if (ok) {
    const size_t plane = (size_t)nx * ny;
    float d[Q];
    pull_node(st + (size_t)b * Q * plane, plane, nx, ny, x, y, d);
    const Moments m = node_moments(d);
    const size_t n = (size_t)b * plane + (size_t)y * nx + x;
    const float dx = m.ux - utx[n], dy = m.uy - uty[n];
    e = dx * dx + dy * dy;
    if (dL_df) {
      const float inv = s / m.rho;
      float *o = dL_df + (size_t)b * Q * plane + (size_t)y * nx + x;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        o[i * plane] = inv * (dx * ((float)cx(i) - m.ux) + dy * ((float)cy(i) - m.uy));
    }
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

// Single block: loss = scale * sum(partials), fixed order (strided then tree).
__global__ void k_sum_partials(const float *__restrict__ partials, int n, float scale,
                               float *loss) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) a += (double)partials[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (float)(red[0] * (double)scale);
}

// ---------------------------------------------------------------------------
// Losses on a node subset S (the training variant of SI section 2): one thread
// per listed node n = b*ny*nx + y*nx + x.  Per-sample errors in FP64, per-block
// FP64 partials (fixed order), then k_sum_partials_f64.  The gradient goes to
// the pre-collision field dL_df (zeroed beforehand by the launcher) with
// atomicAdd: distinct samples touch distinct entries, and a repeated sample
// adds the same value again, so the result does not depend on the order.
// An index outside [0, B ny nx) contributes nothing and sets bad_flag.
// ---------------------------------------------------------------------------
constexpr int SUB_THREADS = 256;

__device__ __forceinline__ bool decode_node(int n, int nx, int ny, int batch, int &x, int &y,
                                            int &b) {
  const long long plane = (long long)nx * ny;
  if (n < 0 || (long long)n >= plane * batch) return false;
  b = (int)(n / plane);
  const int r = (int)(n - (long long)b * plane);
  y = r / nx;
  x = r - y * nx;
  return true;
}

__device__ __forceinline__ void block_sum_f64(double e, double *__restrict__ partials) {
  __shared__ double red[SUB_THREADS];
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = SUB_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// e = |u(n) - u_t(n)|^2 of the pre-collision populations at n;
// dL/df_i(n) = inv_count ((u - u_t).(c_i - u)) / rho   (L = sum e / (2 |S|)).
__global__ void __launch_bounds__(SUB_THREADS)
    k_velocity_loss_subset(const float *__restrict__ st, const int *__restrict__ idx, int count,
                           const float *__restrict__ utx, const float *__restrict__ uty,
                           double *__restrict__ partials, float *__restrict__ dL_df, int nx,
                           int ny, int batch, float inv_count, int *bad_flag) {
  const int s = blockIdx.x * SUB_THREADS + threadIdx.x;
  double e = 0.0;
  if (s < count) {
    int x, y, b;
    if (!decode_node(idx[s], nx, ny, batch, x, y, b)) {
      atomicOr(bad_flag, 1);
    } else {
      const size_t plane = (size_t)nx * ny;
      float d[Q];
      pull_node(st + (size_t)b * Q * plane, plane, nx, ny, x, y, d);
      const Moments m = node_moments(d);
      const size_t n = (size_t)b * plane + (size_t)y * nx + x;
      const float dx = m.ux - utx[n], dy = m.uy - uty[n];
      e = (double)dx * dx + (double)dy * dy;
      if (dL_df) {
        const float inv = inv_count / m.rho;
        float *o = dL_df + (size_t)b * Q * plane + (size_t)y * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i)
          atomicAdd(o + i * plane, inv * (dx * ((float)cx(i) - m.ux) + dy * ((float)cy(i) - m.uy)));
      }
    }
  }
  block_sum_f64(e, partials);
}

// e = sum_i (g_i(n) - t_i(n))^2 with g the stored post-collision populations
// (g_i = state_i + w_i, formed in FP64) and t the target [b][i][y][x];
// dL/dg_i(n) = 2 (g_i - t_i) lands on the pre-collision entry it streams to,
// dL/df_i(n + c_i) (since f_i(x) = g_i(x - c_i)).
__global__ void __launch_bounds__(SUB_THREADS)
    k_population_loss_subset(const float *__restrict__ st, const int *__restrict__ idx, int count,
                             const float *__restrict__ target, double *__restrict__ partials,
                             float *__restrict__ dL_df, int nx, int ny, int batch,
                             int *bad_flag) {
  const int s = blockIdx.x * SUB_THREADS + threadIdx.x;
  double e = 0.0;
  if (s < count) {
    int x, y, b;
    if (!decode_node(idx[s], nx, ny, batch, x, y, b)) {
      atomicOr(bad_flag, 1);
    } else {
      const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
      const size_t at = (size_t)y * nx + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double d = ((double)st[base + i * plane + at] + (double)wf(i)) -
                         (double)target[base + i * plane + at];
        e += d * d;
        if (dL_df) {
          const int xs = wrap_index(x + cx(i), nx), ys = wrap_index(y + cy(i), ny);
          atomicAdd(dL_df + base + i * plane + (size_t)ys * nx + xs, (float)(2.0 * d));
        }
      }
    }
  }
  block_sum_f64(e, partials);
}

// Single block: loss = scale * sum(partials), fixed order (strided then tree).
__global__ void k_sum_partials_f64(const double *__restrict__ partials, int n, double scale,
                                   float *loss) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) a += partials[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (float)(red[0] * scale);
}

// Subsampling filter phi (SI section 2): the coarse node (I, J) takes the fine
// pre-collision populations at (cg I, cg J), f_i = state_i(x - c_i) + w_i.
__global__ void k_subsample(const float *__restrict__ st, float *__restrict__ fc, int nx, int ny,
                            int cg) {
  const int NX = nx / cg, NY = ny / cg;
  const int I = blockIdx.x * NT + threadIdx.x, J = blockIdx.y, b = blockIdx.z;
  if (I >= NX) return;
  const size_t plane = (size_t)nx * ny, cplane = (size_t)NX * NY;
  float d[Q];
  pull_node(st + (size_t)b * Q * plane, plane, nx, ny, I * cg, J * cg, d);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    fc[(size_t)b * Q * cplane + i * cplane + (size_t)J * NX + I] = d[i] + wf(i);
}

// out_i(x) = in_i(x + DIR c_i), DIR = +1 push (transpose of the pull), -1 pull.
template <int DIR>
__global__ void k_shift(const float *__restrict__ in, float *__restrict__ out, int nx, int ny) {
  int x, y, b;
  if (!node_index(nx, x, y, b)) return;
  const size_t plane = (size_t)nx * ny, base = (size_t)b * Q * plane;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrap_index(x + DIR * cx(i), nx), ys = wrap_index(y + DIR * cy(i), ny);
    out[base + i * plane + (size_t)y * nx + x] = in[base + i * plane + (size_t)ys * nx + xs];
  }
}

}  // namespace

cudaError_t launch_step_bgk(const Grid &g, const float *in, float *out, const CollideParams &p,
                            int *flag, cudaStream_t s) {
  return launch_step<KIND_BGK>(g, in, out, p, flag, s);
}

cudaError_t launch_step_smag(const Grid &g, const float *in, float *out, const CollideParams &p,
                             int *flag, cudaStream_t s) {
  return launch_step<KIND_SMAG>(g, in, out, p, flag, s);
}

cudaError_t launch_set_state(const Grid &g, const float *f_pre, float *state, cudaStream_t s) {
  k_set_state<<<node_grid(g), NT, 0, s>>>(f_pre, state, g.nx, g.ny);
  return cudaGetLastError();
}

cudaError_t launch_get_state(const Grid &g, const float *state, float *f_pre, cudaStream_t s) {
  k_get_state<<<node_grid(g), NT, 0, s>>>(state, f_pre, g.nx, g.ny);
  return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const Grid &g, const float *rho, const float *ux,
                                    const float *uy, float *state, cudaStream_t s) {
  k_init_equilibrium<<<node_grid(g), NT, 0, s>>>(rho, ux, uy, state, g.nx, g.ny);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Grid &g, const float *state, float *rho, float *ux, float *uy,
                           cudaStream_t s) {
  k_moments<<<node_grid(g), NT, 0, s>>>(state, rho, ux, uy, g.nx, g.ny);
  return cudaGetLastError();
}

cudaError_t launch_box_filter(const Grid &g, const float *state, int cg, float *f_coarse,
                              cudaStream_t s) {
  dim3 grid((g.nx / cg + NT - 1) / NT, g.ny / cg, g.batch);
  k_box_filter<<<grid, NT, 0, s>>>(state, f_coarse, g.nx, g.ny, cg);
  return cudaGetLastError();
}

int loss_partials(const Grid &g) { return (int)(((g.nx + NT - 1) / NT) * (size_t)g.ny * g.batch); }

cudaError_t launch_velocity_loss(const Grid &g, const float *state, const float *utx,
                                 const float *uty, float *partials, float *loss, float *dL_df,
                                 cudaStream_t s) {
  const float inv_nb = (float)(1.0 / ((double)g.plane() * g.batch));
  k_velocity_loss<<<node_grid(g), NT, 0, s>>>(state, utx, uty, partials, dL_df, g.nx, g.ny,
                                              inv_nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<1, 256, 0, s>>>(partials, loss_partials(g), 0.5f * inv_nb, loss);
  return cudaGetLastError();
}

int subset_partials(int count) { return (count + SUB_THREADS - 1) / SUB_THREADS; }

cudaError_t launch_velocity_loss_subset(const Grid &g, const float *state, const int *idx,
                                        int count, const float *utx, const float *uty,
                                        double *partials, float *loss, float *dL_df,
                                        int *bad_flag, cudaStream_t s) {
  if (dL_df) {
    cudaError_t e = cudaMemsetAsync(dL_df, 0, g.state_floats() * sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  const int blocks = subset_partials(count);
  k_velocity_loss_subset<<<blocks, SUB_THREADS, 0, s>>>(state, idx, count, utx, uty, partials,
                                                        dL_df, g.nx, g.ny, g.batch,
                                                        (float)(1.0 / count), bad_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials_f64<<<1, 256, 0, s>>>(partials, blocks, 0.5 / count, loss);
  return cudaGetLastError();
}

cudaError_t launch_population_loss_subset(const Grid &g, const float *state, const int *idx,
                                          int count, const float *target, double *partials,
                                          float *loss, float *dL_df, int *bad_flag,
                                          cudaStream_t s) {
  if (dL_df) {
    cudaError_t e = cudaMemsetAsync(dL_df, 0, g.state_floats() * sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  const int blocks = subset_partials(count);
  k_population_loss_subset<<<blocks, SUB_THREADS, 0, s>>>(state, idx, count, target, partials,
                                                          dL_df, g.nx, g.ny, g.batch, bad_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials_f64<<<1, 256, 0, s>>>(partials, blocks, 1.0, loss);
  return cudaGetLastError();
}

cudaError_t launch_subsample(const Grid &g, const float *state, int cg, float *f_coarse,
                             cudaStream_t s) {
  dim3 grid((g.nx / cg + NT - 1) / NT, g.ny / cg, g.batch);
  k_subsample<<<grid, NT, 0, s>>>(state, f_coarse, g.nx, g.ny, cg);
  return cudaGetLastError();
}

cudaError_t launch_push(const Grid &g, const float *in, float *out, cudaStream_t s) {
  k_shift<1><<<node_grid(g), NT, 0, s>>>(in, out, g.nx, g.ny);
  return cudaGetLastError();
}

cudaError_t launch_pull(const Grid &g, const float *in, float *out, cudaStream_t s) {
  k_shift<-1><<<node_grid(g), NT, 0, s>>>(in, out, g.nx, g.ny);
  return cudaGetLastError();
}

}  // namespace lbm
