// noalloc.cu -- the velocity loss (lbm_velocity_loss) for callers that may
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// owned up front by its own pool allocator (a framework's caching allocator
// that must not see foreign allocations, or a service whose memory budget is
// partitioned before it starts), or a latency-critical loop where cudaMalloc
// or cudaFree would synchronise the device.  lbm_velocity_loss needs a
// context, and creating one allocates its scratch.  This entry point runs the
// same two kernels (per-block partial sums, then a fixed-order sum) with the
// partial sums kept in a fixed-size array in the library's own device memory.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (4 MiB) until the process exits.  Host code cannot use the
// variable's name as a device address; the first call on each device looks
// the address up with cudaGetSymbolAddress (with that device current) and
// caches it.
#include <mutex>

#include "../../include/lbm.h"
#include "kernels.h"

namespace {

constexpr long long kMaxPartials = 1LL << 20;  // floats: 4 MiB of partial sums
__device__ __align__(256) float g_loss_partials[kMaxPartials];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
float *g_partials_addr[kMaxDevices];  // device address of g_loss_partials, per device

// Address of the scratch array on the current device (looked up once).
int partials_on_current_device(float **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_loss_partials) != cudaSuccess || !p) return LBM_ERR_CUDA;
    g_partials_addr[dev] = static_cast<float *>(p);
  }
  *out = g_partials_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_velocity_loss_noalloc(const float *state, int nx, int ny, int batch,
                                         const float *utx, const float *uty, float *loss,
                                         float *dL_df, void *cuda_stream) {
  if (!state || !utx || !uty || !loss || nx < 1 || ny < 1 || batch < 1) return LBM_ERR_ARG;
  if (ny > 65535 || batch > 65535) return LBM_ERR_ARG;  // gridDim.y / gridDim.z of the launch
  const long long partials = ((long long)nx + 127) / 128 * ny * batch;
  if (partials > kMaxPartials) return LBM_ERR_ARG;  // beyond the fixed scratch array
  float *scratch = nullptr;
  const int rc = partials_on_current_device(&scratch);
  if (rc != LBM_OK) return rc;
  // Every block overwrites its own partial and the final sum reads exactly
  // those, so nothing left by an earlier call needs clearing.
  const lbm::Grid g{nx, ny, batch};
  if (lbm::launch_velocity_loss(g, state, utx, uty, scratch, loss, dL_df,
                                static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return LBM_ERR_CUDA;
  return LBM_OK;
}
