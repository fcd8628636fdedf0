/*
 * lbm3d.h -- C ABI of the paper's own 3D setting in liblbm: a D3Q19
 * lattice-Boltzmann step with BGK, Smagorinsky-BGK and the learned collision
 * with the paper's network, hand-written for sm_103a.
 *
 * Paper: "Kinetic data-driven approach to turbulence subgrid modeling"
 * (arXiv 2403.18466):
 *   - D3Q19 stencil: SI section 1, the D3Q19 velocity stencil table (the
 *     index order below is the table's);
 *   - stream/collide: Eq. S2; BGK: Eq. S3; equilibrium: Eq. S4; EDM forcing:
 *     Eq. S5; Smagorinsky: SI section 1 (same closed form as in lbm.h);
 *   - forcing of the 3D runs: SI section 2, "Definition of the Training
 *     Dataset": F_x(y) = F sin(2 pi m y / ny), F_y(z) = F sin(2 pi m z / nz),
 *     F_z(x) = F sin(2 pi m x / nx) (the paper has m = 1);
 *   - learned collision: SI section 2, "Neural Network Architecture and
 *     Optimization": MLP 19 -> 300 -> 300 -> 100 -> 19 with LeakyReLU (negative
 *     slope 0.01) on the hidden layers and a conservation layer
 *     ohat = o + k1 + k2 c_x + k3 c_y + k4 c_z, k1 = -sum(o)/19,
 *     k_a = -sum(o c_a)/10; post-collision f + (feq - f)/tau + (rho/tau) ohat
 *     + f_ext with input (f - feq)/rho.
 *
 * Conventions (as in lbm.h, which this header includes for the status codes
 * and lbm_collision):
 *   - velocities c_i (x, y, z), i = 0..18:
 *       0:(0,0,0) 1:(-1,0,0) 2:(0,-1,0) 3:(0,0,-1) 4:(0,0,1) 5:(0,1,0) 6:(1,0,0)
 *       7:(-1,-1,0) 8:(-1,0,-1) 9:(-1,0,1) 10:(-1,1,0) 11:(0,-1,-1) 12:(0,-1,1)
 *       13:(0,1,-1) 14:(0,1,1) 15:(1,-1,0) 16:(1,0,-1) 17:(1,0,1) 18:(1,1,0)
 *     weights 1/3 (i = 0), 1/18 (1..6), 1/36 (7..18); c_s^2 = 1/3; dt = dx = 1;
 *   - populations: FP32 [b][i][z][y][x] (x fastest), 19*nx*ny*nz floats per
 *     lattice; density [b][z][y][x]; velocity [b][3][z][y][x];
 *   - device pointers unless named host; caller-owned; asynchronous on the
 *     context's stream; LBM_OK or a negative code; argument errors are found
 *     on the host before any launch; periodic in x, y and z.
 *   - The internal state is the post-collision populations minus the weights
 *     (pull scheme); lbm3d_set_state / lbm3d_get_state convert.
 */
#ifndef LBM3D_H
#define LBM3D_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3d_ctx lbm3d_ctx; /* opaque, library-owned */

typedef struct {
  int nx, ny, nz, batch; /* >= 1 each; ny <= 65535, nz * batch <= 65535 */
  double tau;            /* relaxation time, > 1/2 */
  double smag_cs;        /* Smagorinsky constant, >= 0 (kind LBM_SMAG) */
  double smag_delta;     /* filter width in lattice units, > 0 */
  double force_amp;      /* F of the sine forcing (0 disables it) */
  int force_mode;        /* m of the sine forcing */
  int flags;             /* must be 0 */
} lbm3d_params;

/* The paper's network: w1[300][19], b1[300], w2[300][300], b2[300],
 * w3[100][300], b3[100], w4[19][100], b4[19], row-major [out][in], device
 * pointers, FP32 (dtype 0).  Read at launch, not copied. */
typedef struct {
  const void *w1, *b1, *w2, *b2, *w3, *b3, *w4, *b4;
  int dtype;
} lbm3d_weights;

/* Number of parameters of the packed network (128,319). */
size_t lbm3d_mlp_nparams(void);

/* Host-only: the velocity set and weights as compiled into the kernels
 * (arrays of 19).  Needs no GPU. */
void lbm3d_lattice(int *cx, int *cy, int *cz, float *w);

/* Create a context over two caller-owned device buffers of
 * 19*nx*ny*nz*batch floats each (ping-pong state) on `cuda_stream` (a
 * cudaStream_t, NULL = default stream) of the current device.  Allocates the
 * status flag and the force tables.  LBM_ERR_ARG on bad parameters. */
int lbm3d_init(lbm3d_ctx **out, const lbm3d_params *p, float *f_buf0, float *f_buf1,
               void *cuda_stream);
void lbm3d_destroy(lbm3d_ctx *ctx);

/* Load pre-collision populations (anti-streamed into the internal state) /
 * read the current pre-collision populations. */
int lbm3d_set_state(lbm3d_ctx *ctx, const float *f_pre);
int lbm3d_get_state(lbm3d_ctx *ctx, float *f_pre);

/* Pre-collision state feq(rho, u) (Eq. S4) of rho [b][z][y][x], u [b][3][z][y][x]. */
int lbm3d_init_equilibrium(lbm3d_ctx *ctx, const float *rho, const float *u);

/* Advance n >= 0 steps: pull-stream (Eq. S2), collide with `kind`, EDM force,
 * store.  Both learned kinds take FP32 weights (dtype 0):
 *   LBM_MLP_F32   the network in FP32 on the CUDA cores;
 *   LBM_MLP_BF16  the network on the tensor cores (tcgen05): weights, biases
 *                 and activations rounded to bf16, FP32 accumulation; the
 *                 populations, equilibrium, conservation layer and update
 *                 stay FP32.  The first call allocates 4.6 MB of device
 *                 copies of the weights in operand layout (replicated so that
 *                 the SMs streaming them spread over the L2 cache), refreshed
 *                 at every call.
 * A node reaching |u| >= 0.4 or a non-finite value sets the sticky status
 * flag; a device wait that gives up sets LBM_ERR_TIMEOUT. */
int lbm3d_step(lbm3d_ctx *ctx, int n, lbm_collision kind, const lbm3d_weights *w);

/* rho and u = j/rho of the current pre-collision populations (either NULL). */
int lbm3d_moments(lbm3d_ctx *ctx, float *rho, float *u);

/* Device pointer of the buffer holding the current internal state. */
float *lbm3d_state_buffer(lbm3d_ctx *ctx);

/* Synchronise; LBM_ERR_UNSTABLE / LBM_ERR_TIMEOUT if flagged since the last
 * clear, LBM_ERR_CUDA on a pending CUDA error, else LBM_OK. */
int lbm3d_status(lbm3d_ctx *ctx);
int lbm3d_clear_status(lbm3d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_H */
