// diag.cu -- flow diagnostics of the turbulence statistics the paper reports:
// longitudinal velocity structure functions (SI section 3) and the shell-
// averaged kinetic energy spectrum (main text, energy spectra).
//
// Structure functions: S^p(r) = < [(u(x + r e) - u(x)) . e]^p >, p = 1..6,
// r = 1..rmax, averaged over every node and the two lattice directions
// e = x^, y^ (periodic).  For rmax <= 256: row segments and column strips of
// the field staged in shared memory with an rmax halo, one thread per
// separation; otherwise one block per (r, chunk of rows).  Either way
// per-thread FP32 sums over at most 32 nodes are flushed into FP64
// accumulators and per-block partials are added in a fixed order, so results
// are reproducible.
//
// Energy spectrum: E(k) = 1/2 sum_{round(|k'|) = k} |u_hat(k')|^2 / N^2 for the
// unnormalised 2D DFT (N = nx ny), averaged over the batch, so that the sum
// over all shells is <|u|^2>/2.  The DFT is a cuFFT R2C call; the binning is
// deterministic: shell s collects, in each ky row, the contiguous range of
// kx >= 0 with s^2 - s + 1 <= kx^2 + ky^2 <= s^2 + s, summed by one thread,
// with weight 2 for the kx that stand for their conjugate -kx.
#include <cstdint>
#include <cufft.h>

#include "kernels.h"

namespace lbm {
namespace {

constexpr int SF_THREADS = 256;

__global__ void __launch_bounds__(SF_THREADS)
    k_structure_partials(const float *__restrict__ ux, const float *__restrict__ uy, int nx,
                         int ny, int batch, int rows_per_block, double *__restrict__ part) {
  const int r = blockIdx.x + 1;
  const int chunk = blockIdx.y;
  const int total_rows = ny * batch;
  const int row0 = chunk * rows_per_block;
  const int row1 = min(row0 + rows_per_block, total_rows);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  float facc[6] = {0, 0, 0, 0, 0, 0};
  int pending = 0;
  const size_t N = (size_t)nx * ny;
  for (int row = row0; row < row1; ++row) {
    const int b = row / ny, y = row % ny;
    const int yr = y + r >= ny ? (y + r) % ny : y + r;
    const float *uxr = ux + (size_t)b * N + (size_t)y * nx;
    const float *uyr = uy + (size_t)b * N + (size_t)y * nx;
    const float *uyr2 = uy + (size_t)b * N + (size_t)yr * nx;
    for (int x = threadIdx.x; x < nx; x += SF_THREADS) {
      const int xr = x + r >= nx ? (x + r) % nx : x + r;
      const float dx = uxr[xr] - uxr[x];
      const float dy = uyr2[x] - uyr[x];
      float px = dx, py = dy;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        facc[p] += px + py;
        px *= dx;
        py *= dy;
      }
      if (++pending == 32) {
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          acc[p] += (double)facc[p];
          facc[p] = 0.f;
        }
        pending = 0;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 6; ++p) acc[p] += (double)facc[p];
  __shared__ double red[6][SF_THREADS];
#pragma unroll
  for (int p = 0; p < 6; ++p) red[p][threadIdx.x] = acc[p];
  __syncthreads();
  for (int w = SF_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int p = 0; p < 6; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 6)
    part[((size_t)(r - 1) * gridDim.y + chunk) * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// Tiled form for rmax <= SFT_R (the usual case): one pass over the field per
// direction instead of one per separation.  Thread r - 1 of a block owns
// separation r; the block stages a periodic segment of the field with an rmax
// halo in shared memory, and for every node of it thread r takes
// s[x + r] - s[x] (the first read is a broadcast, the second conflict-free).
// Each thread sums at most 32 terms in FP32 before adding them to its FP64
// sums; each block writes its 6 sums per separation; a last kernel adds the
// blocks in a fixed order.
constexpr int SFT_R = 256;   // separations per block (threads)
constexpr int SFT_X = 1024;  // nodes of a row segment (x direction)
constexpr int SFT_RB = 16;   // rows per x block
constexpr int SFT_C = 32;    // columns of a y strip
constexpr int SFT_Y = 256;   // rows of a y strip
constexpr int SFT_CS = SFT_C + 1;  // padded column stride

struct SfAcc {
  double acc[6];
  float facc[6];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      acc[p] = 0.0;
      facc[p] = 0.f;
    }
  }
  __device__ __forceinline__ void add(float d) {
    const float d2 = d * d, d3 = d2 * d, d4 = d2 * d2;
    facc[0] += d;
    facc[1] += d2;
    facc[2] += d3;
    facc[3] += d4;
    facc[4] += d4 * d;
    facc[5] += d3 * d3;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      acc[p] += (double)facc[p];
      facc[p] = 0.f;
    }
  }
};

__global__ void __launch_bounds__(SFT_R)
    k_sf_rows(const float *__restrict__ ux, int nx, int rows, int rmax, double *__restrict__ part) {
  extern __shared__ float seg[];  // SFT_X + rmax
  const int x0 = blockIdx.x * SFT_X;
  const int w = min(SFT_X, nx - x0);
  const int row0 = blockIdx.y * SFT_RB, row1 = min(row0 + SFT_RB, rows);
  const int r = threadIdx.x + 1;
  SfAcc a;
  a.zero();
  for (int row = row0; row < row1; ++row) {
    const float *u = ux + (size_t)row * nx;  // row b ny + y of the [B][ny][nx] field
    __syncthreads();
    for (int i = threadIdx.x; i < w + rmax; i += SFT_R) seg[i] = u[(x0 + i) % nx];
    __syncthreads();
    if (r <= rmax) {
      for (int xb = 0; xb < w; xb += 32) {
        const int xe = min(xb + 32, w);
        for (int x = xb; x < xe; ++x) a.add(seg[x + r] - seg[x]);
        a.flush();
      }
    }
  }
  if (r <= rmax) {
    double *o = part + ((size_t)(blockIdx.y * gridDim.x + blockIdx.x) * rmax + (r - 1)) * 6;
#pragma unroll
    for (int p = 0; p < 6; ++p) o[p] = a.acc[p];
  }
}

__global__ void __launch_bounds__(SFT_R)
    k_sf_cols(const float *__restrict__ uy, int nx, int ny, int rmax, size_t part_off,
              double *__restrict__ part) {
  extern __shared__ float strip[];  // (SFT_Y + rmax) rows x SFT_CS
  const int x0 = blockIdx.x * SFT_C, cw = min(SFT_C, nx - x0);
  const int y0 = blockIdx.y * SFT_Y, h = min(SFT_Y, ny - y0);
  const float *u = uy + (size_t)blockIdx.z * nx * ny;
  for (int e = threadIdx.x; e < (h + rmax) * SFT_C; e += SFT_R) {
    const int j = e / SFT_C, c = e % SFT_C;
    if (c < cw) strip[j * SFT_CS + c] = u[(size_t)((y0 + j) % ny) * nx + x0 + c];
  }
  __syncthreads();
  const int r = threadIdx.x + 1;
  SfAcc a;
  a.zero();
  if (r <= rmax) {
    for (int j = 0; j < h; ++j) {
      const float *s0 = strip + j * SFT_CS, *s1 = strip + (j + r) * SFT_CS;
      for (int c = 0; c < cw; ++c) a.add(s1[c] - s0[c]);
      a.flush();
    }
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double *o = part + ((part_off + blk) * rmax + (r - 1)) * 6;
#pragma unroll
    for (int p = 0; p < 6; ++p) o[p] = a.acc[p];
  }
}

// S[p][r] = sum over the blocks of the tiled form (in order) / (2 B N)
__global__ void k_sf_final(const double *__restrict__ part, int rmax, int blocks,
                           double inv_count, double *__restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6 * rmax) return;
  const int p = e / rmax, r = e % rmax;
  double s = 0.0;
  for (int k = 0; k < blocks; ++k) s += part[((size_t)k * rmax + r) * 6 + p];
  S[e] = s * inv_count;
}

struct SfTiles {
  int xb, yb;  // blocks along x and y of the row kernel; of the column kernel: bx, by, bz
  int cx, cy, cz;
  __host__ int total() const { return xb * yb + cx * cy * cz; }
};
SfTiles sf_tiles(const Grid &g) {
  SfTiles t;
  t.xb = (g.nx + SFT_X - 1) / SFT_X;
  t.yb = (g.ny * g.batch + SFT_RB - 1) / SFT_RB;
  t.cx = (g.nx + SFT_C - 1) / SFT_C;
  t.cy = (g.ny + SFT_Y - 1) / SFT_Y;
  t.cz = g.batch;
  return t;
}

// S[p][r] = sum over chunks (in order) / (2 B N)
__global__ void k_structure_final(const double *__restrict__ part, int rmax, int chunks,
                                  double inv_count, double *__restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6 * rmax) return;
  const int p = e / rmax, r = e % rmax;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[((size_t)r * chunks + c) * 6 + p];
  S[e] = s * inv_count;
}

__device__ __forceinline__ long long isqrt_floor(long long v) {
  if (v <= 0) return 0;
  long long s = (long long)sqrt((double)v);
  while (s * s > v) --s;
  while ((s + 1) * (s + 1) <= v) ++s;
  return s;
}

// One thread per (ky row j, shell s): sum of the weighted |u_hat|^2 of the row's
// kx range of shell s, for both velocity components and every lattice.
__global__ void k_spectrum_rows(const cufftComplex *__restrict__ uh, int nx, int ny, int batch,
                                int kmax, double *__restrict__ rowpart) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (s > kmax) return;
  const int nxh = nx / 2 + 1;
  const long long ky = j < (ny + 1) / 2 ? j : j - ny;
  const long long lo2 = s == 0 ? 0 : (long long)s * s - s + 1, hi2 = (long long)s * s + s;
  const long long ky2 = ky * ky;
  double acc = 0.0;
  if (hi2 >= ky2) {
    const long long a = lo2 - ky2;
    long long kx_lo = a <= 0 ? 0 : isqrt_floor(a - 1) + 1;  // smallest kx with kx^2 >= a
    long long kx_hi = isqrt_floor(hi2 - ky2);
    if (kx_hi > nxh - 1) kx_hi = nxh - 1;
    for (long long kx = kx_lo; kx <= kx_hi; ++kx) {
      const double wgt = (kx == 0 || (nx % 2 == 0 && kx == nx / 2)) ? 1.0 : 2.0;
      for (int c = 0; c < 2 * batch; ++c) {
        const cufftComplex z = uh[((size_t)c * ny + j) * nxh + kx];
        acc += wgt * ((double)z.x * z.x + (double)z.y * z.y);
      }
    }
  }
  rowpart[(size_t)j * (kmax + 1) + s] = acc;
}

__global__ void k_spectrum_final(const double *__restrict__ rowpart, int ny, int kmax,
                                 double scale, double *__restrict__ E) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > kmax) return;
  double acc = 0.0;
  for (int j = 0; j < ny; ++j) acc += rowpart[(size_t)j * (kmax + 1) + s];
  E[s] = acc * scale;
}

}  // namespace

// The tiled form applies for rmax <= SFT_R and grids within its launch limits.
static bool sf_tiled(const Grid &g, int rmax) {
  const SfTiles t = sf_tiles(g);
  return rmax <= SFT_R && t.yb <= 65535 && t.cy <= 65535 && t.cz <= 65535;
}

size_t structure_partials_doubles(const Grid &g, int rmax) {
  if (sf_tiled(g, rmax)) return (size_t)sf_tiles(g).total() * rmax * 6;
  const int rows = g.ny * g.batch;
  const int rpb = 8;
  const int chunks = (rows + rpb - 1) / rpb;
  return (size_t)rmax * chunks * 6;
}

cudaError_t launch_structure_functions(const Grid &g, const float *ux, const float *uy, int rmax,
                                       double *part, double *S, cudaStream_t s) {
  if (sf_tiled(g, rmax)) {
    const SfTiles t = sf_tiles(g);
    const size_t smem_cols = sizeof(float) * (size_t)(SFT_Y + rmax) * SFT_CS;
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_sf_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(float) * (SFT_Y + SFT_R) * SFT_CS));
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    k_sf_rows<<<dim3(t.xb, t.yb), SFT_R, sizeof(float) * (SFT_X + rmax), s>>>(
        ux, g.nx, g.ny * g.batch, rmax, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sf_cols<<<dim3(t.cx, t.cy, t.cz), SFT_R, smem_cols, s>>>(uy, g.nx, g.ny, rmax,
                                                              (size_t)t.xb * t.yb, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sf_final<<<(6 * rmax + 255) / 256, 256, 0, s>>>(part, rmax, t.total(),
                                                      1.0 / (2.0 * (double)g.nodes()), S);
    return cudaGetLastError();
  }
  const int rows = g.ny * g.batch;
  const int rpb = 8;
  const int chunks = (rows + rpb - 1) / rpb;
  if (chunks > 65535) return cudaErrorInvalidValue;
  k_structure_partials<<<dim3(rmax, chunks), SF_THREADS, 0, s>>>(ux, uy, g.nx, g.ny, g.batch, rpb,
                                                                  part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_structure_final<<<(6 * rmax + 255) / 256, 256, 0, s>>>(part, rmax, chunks,
                                                           1.0 / (2.0 * (double)g.nodes()), S);
  return cudaGetLastError();
}

size_t spectrum_rowpart_doubles(const Grid &g, int kmax) { return (size_t)g.ny * (kmax + 1); }

// u: [2B][ny][nx] real (ux of every lattice, then uy); uh: [2B][ny][nx/2+1].
cudaError_t launch_energy_spectrum(const Grid &g, float *u, void *uh, void **plan_io, int kmax,
                                   double *rowpart, double *E, cudaStream_t s) {
  cufftHandle plan;
  if (!*plan_io) {
    int n[2] = {g.ny, g.nx};
    if (cufftPlanMany(&plan, 2, n, nullptr, 1, g.ny * g.nx, nullptr, 1, g.ny * (g.nx / 2 + 1),
                      CUFFT_R2C, 2 * g.batch) != CUFFT_SUCCESS)
      return cudaErrorUnknown;
    *plan_io = reinterpret_cast<void *>(static_cast<uintptr_t>(plan) + 1);
  }
  plan = static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(*plan_io) - 1);
  if (cufftSetStream(plan, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
  if (cufftExecR2C(plan, u, static_cast<cufftComplex *>(uh)) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  dim3 grid((kmax + 1 + 127) / 128, g.ny);
  k_spectrum_rows<<<grid, 128, 0, s>>>(static_cast<const cufftComplex *>(uh), g.nx, g.ny,
                                       g.batch, kmax, rowpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double N = (double)g.nx * g.ny;
  k_spectrum_final<<<(kmax + 1 + 127) / 128, 128, 0, s>>>(rowpart, g.ny, kmax,
                                                          0.5 / (N * N * g.batch), E);
  return cudaGetLastError();
}

void destroy_spectrum_plan(void *plan_io) {
  if (plan_io) cufftDestroy(static_cast<cufftHandle>(reinterpret_cast<uintptr_t>(plan_io) - 1));
}

}  // namespace lbm
