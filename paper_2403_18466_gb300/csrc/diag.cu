// diag.cu -- flow diagnostics of the turbulence statistics the paper reports:
// longitudinal velocity structure functions (SI section 3) and the shell-
// averaged kinetic energy spectrum (main text, energy spectra).
//
// Structure functions: S^p(r) = < [(u(x + r e) - u(x)) . e]^p >, p = 1..6,
// r = 1..rmax, averaged over every node and the two lattice directions
// e = x^, y^ (periodic).  One block per (r, chunk of rows); per-thread FP32
// sums over at most 32 nodes are flushed into FP64 accumulators; per-block
// partials are added in a fixed order, so results are reproducible.
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

size_t structure_partials_doubles(const Grid &g, int rmax) {
  const int rows = g.ny * g.batch;
  const int rpb = 8;
  const int chunks = (rows + rpb - 1) / rpb;
  return (size_t)rmax * chunks * 6;
}

cudaError_t launch_structure_functions(const Grid &g, const float *ux, const float *uy, int rmax,
                                       double *part, double *S, cudaStream_t s) {
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
