// kernels.h -- internal launcher interface between the C ABI (lbm_api.cu)
// and the kernel translation units.  Not installed; not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace lbm {

// Grid description shared by all launchers.
struct Grid {
  int nx, ny, batch;
  size_t plane() const { return (size_t)nx * ny; }
  size_t nodes() const { return plane() * batch; }
  size_t state_floats() const { return 9 * nodes(); }
};

// Per-launch collision parameters (FP32 copies of lbm_params).
struct CollideParams {
  float tau, omega;      // tau, 1/tau
  float tau0_sq;         // tau^2 (Smagorinsky)
  float smag_c18;        // 18 (C_s Delta)^2 (Smagorinsky)
  const float *force;    // per-row F_x(y), ny floats (device), or nullptr
};

// FP32 weights packed in the library's order (device pointers).
struct MlpF32 {
  const float *w1, *b1, *w2, *b2, *w3, *b3;
};

// step_fp32.cu ---------------------------------------------------------------
cudaError_t launch_step_bgk(const Grid &g, const float *in, float *out, const CollideParams &p,
                            int *flag, cudaStream_t s);
cudaError_t launch_step_smag(const Grid &g, const float *in, float *out, const CollideParams &p,
                             int *flag, cudaStream_t s);
cudaError_t launch_set_state(const Grid &g, const float *f_pre, float *state, cudaStream_t s);
cudaError_t launch_get_state(const Grid &g, const float *state, float *f_pre, cudaStream_t s);
cudaError_t launch_init_equilibrium(const Grid &g, const float *rho, const float *ux,
                                    const float *uy, float *state, cudaStream_t s);
cudaError_t launch_moments(const Grid &g, const float *state, float *rho, float *ux, float *uy,
                           cudaStream_t s);
cudaError_t launch_box_filter(const Grid &g, const float *state, int cg, float *f_coarse,
                              cudaStream_t s);
// Loss: per-block partial sums into `partials` (>= loss_partials(g) floats),
// then a single-block fixed-order sum into loss[0].
int loss_partials(const Grid &g);
cudaError_t launch_velocity_loss(const Grid &g, const float *state, const float *utx,
                                 const float *uty, float *partials, float *loss, float *dL_df,
                                 cudaStream_t s);
// Subset losses: per-block FP64 partials into `partials` (>= subset_partials(count)
// doubles), then a single-block fixed-order sum into loss[0].  dL_df (nullable)
// is zeroed and receives the gradient w.r.t. the pre-collision populations.
int subset_partials(int count);
cudaError_t launch_velocity_loss_subset(const Grid &g, const float *state, const int *idx,
                                        int count, const float *utx, const float *uty,
                                        double *partials, float *loss, float *dL_df,
                                        int *bad_flag, cudaStream_t s);
cudaError_t launch_population_loss_subset(const Grid &g, const float *state, const int *idx,
                                          int count, const float *target, double *partials,
                                          float *loss, float *dL_df, int *bad_flag,
                                          cudaStream_t s);
cudaError_t launch_subsample(const Grid &g, const float *state, int cg, float *f_coarse,
                             cudaStream_t s);
// push (transpose of the pull) of an adjoint field: out_i(x) = in_i(x + c_i)
cudaError_t launch_push(const Grid &g, const float *in, float *out, cudaStream_t s);
// pull of an adjoint field: out_i(x) = in_i(x - c_i)
cudaError_t launch_pull(const Grid &g, const float *in, float *out, cudaStream_t s);

// mlp_f32.cu -------------------------------------------------------------------
cudaError_t launch_step_mlp_f32(const Grid &g, const float *in, float *out,
                                const CollideParams &p, const MlpF32 &w, int *flag,
                                cudaStream_t s);

// mlp_bf16.cu ------------------------------------------------------------------
// weights: FP32 (dtype 0) or BF16 (dtype 1), same packed row-major layout.
// wait_limit: polls of each bounded mbarrier wait before the kernel gives up
// and sets *timeout_flag (0 = the default, 2^20); max_ctas: cap on the
// persistent grid (0 = one CTA per SM); chain: the previous operation on `s`
// is this kernel with the same weights, so it is launched as a programmatic
// dependent of it (its prologue overlaps that kernel's last tiles).
cudaError_t launch_step_mlp_bf16(const Grid &g, const float *in, float *out,
                                 const CollideParams &p, const void *const wptr[6], int dtype,
                                 int *flag, int *timeout_flag, cudaStream_t s,
                                 unsigned wait_limit = 0, int max_ctas = 0, bool chain = false);

// Compiled layout of the tensor-core step: tile warpgroups per SM and, of
// every 8 activation pairs, how many the XU evaluates.
void mlp_bf16_layout(int *warpgroups, int *xu_pairs_per_8);
// The step kernel's activations element-wise (0: XU path, 1: FMA path as
// stored, 2: FMA path before its bf16 rounding).
cudaError_t launch_activation(const float *a, int n, int path, float *out, cudaStream_t s);

// adjoint.cu -------------------------------------------------------------------
// Number of CTAs (= rows of per-CTA dW partials) of the adjoint step.
int adjoint_blocks(const Grid &g, int sms);
size_t adjoint_smem_bytes();
cudaError_t launch_adjoint_step(const Grid &g, const float *state_n, const float *lam_next,
                                float *lam_out, const CollideParams &p, const MlpF32 &w,
                                float *dw_partials, int rows, int accumulate, cudaStream_t s);
cudaError_t launch_reduce_dw(const float *dw_partials, int rows, float *dW, cudaStream_t s);

// adjoint_tc.cu ----------------------------------------------------------------
// Tensor-core adjoint step (BF16 operands, FP32 accumulation); one partial row
// per CTA (one persistent CTA per SM).  Launched as a programmatic dependent
// of the previous kernel on `s`, which must not write the weights `w` (its
// prologue reads them before waiting for that kernel).
int adjoint_tc_rows(const Grid &g, int sms);
cudaError_t launch_adjoint_tc(const Grid &g, const float *state_n, const float *lam_next,
                              float *lam_out, const CollideParams &p, const MlpF32 &w,
                              float *dw_partials, int rows, int accumulate, int *timeout_flag,
                              cudaStream_t s);

// diag.cu ----------------------------------------------------------------------
size_t structure_partials_doubles(const Grid &g, int rmax);
cudaError_t launch_structure_functions(const Grid &g, const float *ux, const float *uy, int rmax,
                                       double *part, double *S, cudaStream_t s);
size_t spectrum_rowpart_doubles(const Grid &g, int kmax);
// u: [2B][ny][nx] (ux of every lattice, then uy), uh: complex [2B][ny][nx/2+1];
// *plan_io caches the FFT plan (created on first use).
cudaError_t launch_energy_spectrum(const Grid &g, float *u, void *uh, void **plan_io, int kmax,
                                   double *rowpart, double *E, cudaStream_t s);
void destroy_spectrum_plan(void *plan_io);

}  // namespace lbm
