// kernels3d.h -- internal launcher interface of the D3Q19 kernels (the paper's
// 3D setting) for the C ABI in lbm3d_api.cu.  Not installed; not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace lbm {
namespace d3 {

struct Grid3 {
  int nx, ny, nz, batch;
  __host__ __device__ size_t volume() const { return (size_t)nx * ny * nz; }
  size_t nodes() const { return volume() * batch; }
  size_t state_floats() const { return 19 * nodes(); }
};

// FP32 copies of the collision parameters; force tables are per-axis sines
// (F_x(y), F_y(z), F_z(x)), device arrays of ny, nz, nx floats, or nullptr.
struct Collide3 {
  float tau, omega, tau0_sq, smag_c18;
  const float *fx_y, *fy_z, *fz_x;
};

// FP32 weights of the paper's network in the packed order (device pointers).
struct Mlp3 {
  const float *w1, *b1, *w2, *b2, *w3, *b3, *w4, *b4;
};

// d3q19_step.cu
cudaError_t launch_step(const Grid3 &g, const float *in, float *out, const Collide3 &c, int kind,
                        int *flag, cudaStream_t s);
size_t mlp_f32_smem_bytes();
cudaError_t launch_step_mlp_f32(const Grid3 &g, const float *in, float *out, const Collide3 &c,
                                const Mlp3 &w, int *flag, cudaStream_t s);
cudaError_t launch_set_state(const Grid3 &g, const float *f_pre, float *state, cudaStream_t s);

// d3q19_mlp_tc.cu: the tensor-core learned collision.  The FP32 weights are
// first laid out as BF16 operand tiles in a device buffer of
// mlp_tc_weight_bytes() bytes (launch_prepare_weights_tc), which the step
// kernel reads (resident W1/W4, streamed W2/W3).  One persistent CTA per SM.
size_t mlp_tc_weight_bytes();
cudaError_t launch_prepare_weights_tc(const Mlp3 &w, void *gw, cudaStream_t s);
cudaError_t launch_step_mlp_tc(const Grid3 &g, const float *in, float *out, const Collide3 &c,
                               const void *gw, int sms, int *flag, int *timeout_flag,
                               cudaStream_t s);
cudaError_t launch_get_state(const Grid3 &g, const float *state, float *f_pre, cudaStream_t s);
cudaError_t launch_init_equilibrium(const Grid3 &g, const float *rho, const float *u,
                                    float *state, cudaStream_t s);
cudaError_t launch_moments(const Grid3 &g, const float *state, float *rho, float *u,
                           cudaStream_t s);

}  // namespace d3
}  // namespace lbm
