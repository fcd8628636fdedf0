// d3q19_step.cu -- the paper's 3D setting on the CUDA cores: the fused D3Q19
// pull-stream + BGK / Smagorinsky-BGK step with the paper's three-component sine
// forcing (EDM, Eq. S5), the FP32 learned collision with the paper's network
// (19 -> 300 -> 300 -> 100 -> 19, LeakyReLU, conservation layer with kappa
// denominators 19 and 10), and the data-movement kernels around them.
//
// Step kernels: one thread per node along x; each pulls f_i(x) = g_i(x - c_i)
// (periodic) from the previous buffer, collides and stores at x.  Algorithmic
// traffic 76 B read + 76 B written per node.
//
// FP32 learned collision: a block of 128 threads owns 32 nodes of one x row;
// every layer's activations of those nodes live in shared memory as [k][node]
// (conflict-free column reads), and each warp computes a quarter of the layer's
// outputs for all 32 nodes, reading weight rows with warp-uniform loads.
#include "d3q19.cuh"
#include "kernels3d.h"
#include "umma.cuh"

namespace lbm {
namespace d3 {
namespace {

constexpr int NT = 128;
enum { KIND_BGK = 0, KIND_SMAG = 1 };

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

struct Pos {
  int x, y, z, b;
};

__device__ __forceinline__ bool node_pos(const Grid3 &g, Pos &p) {
  p.x = blockIdx.x * NT + threadIdx.x;
  p.y = blockIdx.y;
  p.z = blockIdx.z % g.nz;
  p.b = blockIdx.z / g.nz;
  return p.x < g.nx;
}

__device__ __forceinline__ void pull(const float *__restrict__ in, const Grid3 &g, const Pos &p,
                                     float d[Q]) {
  const size_t vol = g.volume();
  const float *gb = in + (size_t)p.b * Q * vol;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrapi(p.x - cx(i), g.nx), ys = wrapi(p.y - cy(i), g.ny),
              zs = wrapi(p.z - cz(i), g.nz);
    d[i] = __ldg(gb + (size_t)i * vol + ((size_t)zs * g.ny + ys) * g.nx + xs);
  }
}

__device__ __forceinline__ size_t at(const Grid3 &g, const Pos &p) {
  return ((size_t)p.z * g.ny + p.y) * g.nx + p.x;
}

__device__ __forceinline__ void node_force(const Collide3 &c, const Pos &p, float &Fx, float &Fy,
                                           float &Fz) {
  Fx = c.fx_y ? c.fx_y[p.y] : 0.f;
  Fy = c.fy_z ? c.fy_z[p.z] : 0.f;
  Fz = c.fz_x ? c.fz_x[p.x] : 0.f;
}

__device__ __forceinline__ void flag_bad(bool bad, int *flag) {
  const unsigned mask = __ballot_sync(__activemask(), bad);
  if (mask && (threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
    if (*reinterpret_cast<volatile int *>(flag) == 0) atomicOr(flag, 1);
  }
}

template <int KIND>
__global__ void __launch_bounds__(NT) k3_step(const float *__restrict__ in, float *__restrict__ out,
                                              Grid3 g, Collide3 c, int *flag) {
  umma::griddep_wait();  // launched as a dependent of the previous step
  umma::griddep_launch_dependents();
  Pos p;
  if (!node_pos(g, p)) return;
  float d[Q], deq[Q];
  pull(in, g, p, d);
  const Moments m = node_moments(d);
  shifted_feq(m, deq);
  const float om = KIND == KIND_SMAG ? smag_omega(d, deq, m.inv_rho, c.tau0_sq, c.tau, c.smag_c18)
                                     : c.omega;
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] += om * (deq[i] - d[i]);
  float Fx, Fy, Fz;
  node_force(c, p, Fx, Fy, Fz);
  add_edm_force(m, Fx, Fy, Fz, d);
  flag_bad(is_unstable(m), flag);
  const size_t vol = g.volume();
  float *o = out + (size_t)p.b * Q * vol + at(g, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) o[(size_t)i * vol] = d[i];
}

// ---------------------------------------------------------------------------
// FP32 learned collision.
// ---------------------------------------------------------------------------
constexpr int MT = 128;     // threads
constexpr int MN = 32;      // nodes per block
constexpr int MW = MT / 32; // warps

// y[j][n] = act(b[j] + sum_k W[j][k] x[k][n]) for j = warp, warp + MW, ...
template <bool ACT>
__device__ __forceinline__ void dense_layer(const float *__restrict__ W, const float *__restrict__ b,
                                            int nout, int nin, const float *x, float *y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < nout; j += MW) {
    const float *wr = W + (size_t)j * nin;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int k = 0;
    for (; k + 4 <= nin; k += 4) {
      a0 = fmaf(__ldg(wr + k), x[(k + 0) * MN + lane], a0);
      a1 = fmaf(__ldg(wr + k + 1), x[(k + 1) * MN + lane], a1);
      a2 = fmaf(__ldg(wr + k + 2), x[(k + 2) * MN + lane], a2);
      a3 = fmaf(__ldg(wr + k + 3), x[(k + 3) * MN + lane], a3);
    }
    for (; k < nin; ++k) a0 = fmaf(__ldg(wr + k), x[k * MN + lane], a0);
    float a = __ldg(b + j) + ((a0 + a1) + (a2 + a3));
    if (ACT) a = a >= 0.f ? a : LEAKY * a;
    y[j * MN + lane] = a;
  }
}

struct MlpSmem {
  float x[Q * MN];
  float h1[H1 * MN];
  float h2[H2 * MN];
  float h3[H3 * MN];
  float o[Q * MN];
};

__global__ void __launch_bounds__(MT) k3_step_mlp_f32(const float *__restrict__ in,
                                                      float *__restrict__ out, Grid3 g, Collide3 c,
                                                      Mlp3 w, int *flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // block -> (row, 32-node segment); every warp loads the same 32 nodes
  const int segs = (g.nx + MN - 1) / MN;
  const int seg = blockIdx.x % segs;
  const int row = blockIdx.x / segs;  // over (b, z, y)
  Pos p;
  p.x = seg * MN + lane;
  p.y = row % g.ny;
  p.z = (row / g.ny) % g.nz;
  p.b = row / (g.ny * g.nz);
  const bool live = p.x < g.nx;
  float d[Q], deq[Q];
  Moments m;
  m.drho = 0.f;
  m.rho = 1.f;
  m.ux = m.uy = m.uz = 0.f;
  if (live) {
    pull(in, g, p, d);
    m = node_moments(d);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = 0.f;
  }
  shifted_feq(m, deq);
  if (warp == 0) {
    const float inv = 1.0f / m.rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) s.x[i * MN + lane] = (d[i] - deq[i]) * inv;
  }
  __syncthreads();
  dense_layer<true>(w.w1, w.b1, H1, Q, s.x, s.h1);
  __syncthreads();
  dense_layer<true>(w.w2, w.b2, H2, H1, s.h1, s.h2);
  __syncthreads();
  dense_layer<true>(w.w3, w.b3, H3, H2, s.h2, s.h3);
  __syncthreads();
  dense_layer<false>(w.w4, w.b4, Q, H3, s.h3, s.o);
  __syncthreads();
  if (warp != 0 || !live) return;
  float o[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) o[i] = s.o[i * MN + lane];
  project(o);
  const float scale = m.rho * c.omega;
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] += c.omega * (deq[i] - d[i]) + scale * o[i];
  float Fx, Fy, Fz;
  node_force(c, p, Fx, Fy, Fz);
  add_edm_force(m, Fx, Fy, Fz, d);
  flag_bad(is_unstable(m), flag);
  const size_t vol = g.volume();
  float *op = out + (size_t)p.b * Q * vol + at(g, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) op[(size_t)i * vol] = d[i];
}

// state_i(x) = f_i(x + c_i) - w_i (anti-streaming into the pull representation)
__global__ void k3_set_state(const float *__restrict__ f, float *__restrict__ st, Grid3 g) {
  Pos p;
  if (!node_pos(g, p)) return;
  const size_t vol = g.volume(), base = (size_t)p.b * Q * vol;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrapi(p.x + cx(i), g.nx), ys = wrapi(p.y + cy(i), g.ny),
              zs = wrapi(p.z + cz(i), g.nz);
    st[base + (size_t)i * vol + at(g, p)] =
        f[base + (size_t)i * vol + ((size_t)zs * g.ny + ys) * g.nx + xs] - wf(i);
  }
}

// f_i(x) = state_i(x - c_i) + w_i
__global__ void k3_get_state(const float *__restrict__ st, float *__restrict__ f, Grid3 g) {
  Pos p;
  if (!node_pos(g, p)) return;
  float d[Q];
  pull(st, g, p, d);
  const size_t vol = g.volume(), base = (size_t)p.b * Q * vol;
#pragma unroll
  for (int i = 0; i < Q; ++i) f[base + (size_t)i * vol + at(g, p)] = d[i] + wf(i);
}

// feq(rho, u) at x becomes the pre-collision state: written to x - c_i.
__global__ void k3_init_equilibrium(const float *__restrict__ rho, const float *__restrict__ u,
                                    float *__restrict__ st, Grid3 g) {
  Pos p;
  if (!node_pos(g, p)) return;
  const size_t vol = g.volume(), base = (size_t)p.b * Q * vol;
  const size_t n = at(g, p);
  Moments m;
  m.rho = rho[(size_t)p.b * vol + n];
  m.drho = m.rho - 1.0f;
  m.ux = u[((size_t)p.b * 3 + 0) * vol + n];
  m.uy = u[((size_t)p.b * 3 + 1) * vol + n];
  m.uz = u[((size_t)p.b * 3 + 2) * vol + n];
  float deq[Q];
  shifted_feq(m, deq);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int xs = wrapi(p.x - cx(i), g.nx), ys = wrapi(p.y - cy(i), g.ny),
              zs = wrapi(p.z - cz(i), g.nz);
    st[base + (size_t)i * vol + ((size_t)zs * g.ny + ys) * g.nx + xs] = deq[i];
  }
}

// rho [b][z][y][x] and u [b][3][z][y][x] of the pre-collision populations
__global__ void k3_moments(const float *__restrict__ st, float *rho, float *u, Grid3 g) {
  Pos p;
  if (!node_pos(g, p)) return;
  float d[Q];
  pull(st, g, p, d);
  const Moments m = node_moments(d);
  const size_t vol = g.volume(), n = at(g, p);
  if (rho) rho[(size_t)p.b * vol + n] = m.rho;
  if (u) {
    u[((size_t)p.b * 3 + 0) * vol + n] = m.ux;
    u[((size_t)p.b * 3 + 1) * vol + n] = m.uy;
    u[((size_t)p.b * 3 + 2) * vol + n] = m.uz;
  }
}

dim3 node_grid(const Grid3 &g) { return dim3((g.nx + NT - 1) / NT, g.ny, g.nz * g.batch); }

}  // namespace

// Programmatic dependent launch: the kernel waits for the previous kernel on
// the stream before its first global access, which hides the launch gap.
cudaError_t launch_step(const Grid3 &g, const float *in, float *out, const Collide3 &c, int kind,
                        int *flag, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = node_grid(g);
  cfg.blockDim = dim3(NT);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (kind == KIND_SMAG) return cudaLaunchKernelEx(&cfg, k3_step<KIND_SMAG>, in, out, g, c, flag);
  return cudaLaunchKernelEx(&cfg, k3_step<KIND_BGK>, in, out, g, c, flag);
}

size_t mlp_f32_smem_bytes() { return sizeof(MlpSmem); }

cudaError_t launch_step_mlp_f32(const Grid3 &g, const float *in, float *out, const Collide3 &c,
                                const Mlp3 &w, int *flag, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k3_step_mlp_f32,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(MlpSmem));
  if (e != cudaSuccess) return e;
  const size_t rows = (size_t)g.ny * g.nz * g.batch;
  const size_t blocks = rows * ((g.nx + MN - 1) / MN);
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  k3_step_mlp_f32<<<(unsigned)blocks, MT, sizeof(MlpSmem), s>>>(in, out, g, c, w, flag);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const Grid3 &g, const float *f_pre, float *state, cudaStream_t s) {
  k3_set_state<<<node_grid(g), NT, 0, s>>>(f_pre, state, g);
  return cudaGetLastError();
}

cudaError_t launch_get_state(const Grid3 &g, const float *state, float *f_pre, cudaStream_t s) {
  k3_get_state<<<node_grid(g), NT, 0, s>>>(state, f_pre, g);
  return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const Grid3 &g, const float *rho, const float *u,
                                    float *state, cudaStream_t s) {
  k3_init_equilibrium<<<node_grid(g), NT, 0, s>>>(rho, u, state, g);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Grid3 &g, const float *state, float *rho, float *u,
                           cudaStream_t s) {
  k3_moments<<<node_grid(g), NT, 0, s>>>(state, rho, u, g);
  return cudaGetLastError();
}

}  // namespace d3
}  // namespace lbm
