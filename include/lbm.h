/*
 * lbm.h -- C ABI of liblbm: a D2Q9 lattice-Boltzmann step with BGK,
 * Smagorinsky-BGK and learned (MLP) collisions, its adjoint, and the data
 * pipeline kernels, hand-written for sm_103a.
 *
 * Paper: "Kinetic data-driven approach to turbulence subgrid modeling"
 * (arXiv 2403.18466).  The operations follow its statement of the method:
 *   - lattice Boltzmann equation, stream/collide split: Methods, Eq. S2;
 *   - BGK collision: Eq. S3; equilibrium: Eq. S4; EDM forcing: Eq. S5;
 *   - Smagorinsky relaxation time: SI section 1 (Eq. S7 and the strain
 *     from the non-equilibrium stress, read with the Chapman-Enskog relation
 *     S = -Pi_neq / (2 rho cs^2 tau_eff), which gives the local closed form
 *     tau_eff = (tau0 + sqrt(tau0^2 + 18 (C_s Delta)^2 Q / rho)) / 2,
 *     Q = sqrt(2 Pi_neq : Pi_neq));
 *   - learned collision with mass/momentum projection: Eqs. S10-S12;
 *   - unrolled training and its loss: SI section 2, Eq. S13;
 *   - coarse-graining filter and rescaled tau: SI section 2, Eq. S9.
 *
 * Conventions common to every entry point
 *   - D2Q9 velocities, in this order (index: c_x, c_y):
 *       0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
 *     weights 4/9 (i=0), 1/9 (i=1..4), 1/36 (i=5..8); c_s^2 = 1/3; dt = dx = 1.
 *   - Population arrays are FP32 structure-of-arrays, index [b][i][y][x]
 *     (x fastest), plane stride nx*ny, batch stride 9*nx*ny.  Scalar fields
 *     (rho, u_x, u_y, targets) are [b][y][x].
 *   - All array pointers are DEVICE pointers unless the name says host.
 *     The caller owns every array it passes; the library never frees them.
 *   - Every call is asynchronous on the context's stream unless documented
 *     otherwise, and returns LBM_OK (0) or a negative LBM_ERR_* code.
 *     Nothing throws across the ABI.  Argument errors are detected on the
 *     host before any launch.
 *   - Periodic boundaries in x and y.
 *   - Kolmogorov body force F = (F0 sin(2 pi m y / ny), 0), applied by EDM
 *     after the collision at every step of every kind (F0 = 0 disables it).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)         /* invalid argument (null pointer, size, kind) */
#define LBM_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define LBM_ERR_UNSUPPORTED (-3) /* valid but not supported by this library */
#define LBM_ERR_UNSTABLE (-4)    /* a node reached |u| >= 0.4 or a non-finite value */
#define LBM_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

typedef enum {
  LBM_BGK = 0,      /* Eq. S3 */
  LBM_SMAG = 1,     /* Smagorinsky-BGK, SI section 1 */
  LBM_MLP_BF16 = 2, /* Eq. S10, MLP on the tensor cores (BF16 in, FP32 accumulate) */
  LBM_MLP_F32 = 3   /* Eq. S10, MLP in FP32 on the CUDA cores */
} lbm_collision;

typedef struct {
  int nx, ny, batch;   /* grid and number of independent lattices (>= 1 each;
                          ny, batch <= 65535; nx*ny <= 2^31 - 1;
                          ceil(nx/128)*ny*batch <= 2^31 - 1; 9*nx*ny*batch <= 2^40;
                          lbm_init returns LBM_ERR_ARG beyond these) */
  double tau;          /* relaxation time, > 0.5 (Eq. S3, S6) */
  double smag_cs;      /* Smagorinsky constant C_s (used by LBM_SMAG) */
  double smag_delta;   /* filter width Delta in lattice units (LBM_SMAG) */
  double force_amp;    /* Kolmogorov amplitude F0 */
  int force_mode;      /* Kolmogorov wavenumber m */
  int flags;           /* reserved, must be 0 */
} lbm_params;

/* MLP 9 -> 64 -> 64 -> 9, tanh hidden layers, linear output (Eq. S10 network
 * with this library's widths).  Device pointers, row-major [out][in]:
 * w1[64][9], b1[64], w2[64][64], b2[64], w3[9][64], b3[9].
 * dtype 0 = FP32 (both MLP kinds), 1 = BF16 (LBM_MLP_BF16 only).  The
 * weights are read at launch, never copied or retained. */
typedef struct {
  const void *w1, *b1, *w2, *b2, *w3, *b3;
  int dtype;
} lbm_weights;

#define LBM_MLP_HIDDEN 64
#define LBM_MLP_NPARAMS 5385 /* packed order w1, b1, w2, b2, w3, b3 */

/* Create a context over two caller-owned device state buffers of
 * 9*nx*ny*batch floats each (ping-pong), on `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream).  The buffers hold the library's internal
 * state representation: post-collision populations minus the weights w_i
 * (the pull scheme stores f_post at time t; the pre-collision populations
 * at t+1 are the streamed values).  Use lbm_set_state / lbm_get_state to
 * move populations in and out.  Allocates the context and a small device
 * scratch area (status flag, force table, reduction partials), freed by
 * lbm_destroy.  Synchronous. */
int lbm_init(lbm_ctx **out, const lbm_params *p, float *f_buf0, float *f_buf1,
             void *cuda_stream);

/* Release the context and its scratch (not the caller's buffers). */
void lbm_destroy(lbm_ctx *ctx);

/* Load pre-collision populations f_pre [b][i][y][x] (unshifted) as the
 * current state.  Anti-streams them (SI section 2, step 4) into the current
 * buffer. */
int lbm_set_state(lbm_ctx *ctx, const float *f_pre);

/* Write the current pre-collision populations (streamed, unshifted) to
 * f_pre [b][i][y][x]. */
int lbm_get_state(lbm_ctx *ctx, float *f_pre);

/* Set the state to the equilibrium feq(rho, u) (Eq. S4) of the given fields
 * [b][y][x] as pre-collision populations. */
int lbm_init_equilibrium(lbm_ctx *ctx, const float *rho, const float *ux, const float *uy);

/* Advance n >= 0 steps: per node, pull-stream (Eq. S2), collide with `kind`
 * (Eq. S3 / SI sec. 1 / Eq. S10-S12), add the EDM force (Eq. S5), store.
 * `w` is required for the MLP kinds and ignored otherwise.  A node whose
 * velocity reaches |u| >= 0.4, or becomes non-finite, sets the sticky
 * status flag read by lbm_status. */
int lbm_step(lbm_ctx *ctx, int n, lbm_collision kind, const lbm_weights *w);

/* Density and velocity u = j / rho of the current pre-collision populations
 * into rho, ux, uy [b][y][x] (any of them may be NULL). */
int lbm_moments(lbm_ctx *ctx, float *rho, float *ux, float *uy);

/* Device pointer of the buffer holding the current state (internal
 * representation, see lbm_init), or NULL. */
float *lbm_state_buffer(lbm_ctx *ctx);

/* Synchronise the stream and return LBM_ERR_UNSTABLE if any step since the
 * last lbm_clear_status flagged a node, LBM_ERR_TIMEOUT if a kernel gave up a
 * bounded wait, LBM_ERR_ARG if a subset loss met a node index out of range, a
 * pending CUDA error as LBM_ERR_CUDA, else LBM_OK.  Synchronous. */
int lbm_status(lbm_ctx *ctx);
int lbm_clear_status(lbm_ctx *ctx);

/* Failure detection (no counterpart in the paper): the tensor-core step
 * kernel waits for each of its GEMMs with a bounded number of mbarrier polls
 * and, when a wait runs out, stops, frees its tensor memory and sets the
 * status that lbm_status reports as LBM_ERR_TIMEOUT (the state written by
 * that step is then incomplete).  This sets the number of polls per wait for
 * the later lbm_step calls of this context; 0 restores the default (2^20,
 * far above any real GEMM latency).  A small value lets a test make a wait
 * run out on purpose; the kernel's final wait for its own outstanding GEMM
 * always uses the default, so tensor memory is never released under a GEMM
 * in flight.  Host-side only; LBM_ERR_ARG for a NULL context. */
int lbm_set_wait_limit(lbm_ctx *ctx, unsigned polls);

/* Launch shape of the tensor-core step (no counterpart in the paper): caps
 * the persistent grid of LBM_MLP_BF16 steps at n CTAs for the later lbm_step
 * calls of this context (0, the default, restores one CTA per SM).  With
 * fewer CTAs each warpgroup walks more tiles, so a lattice small enough for
 * an element-by-element check against a reference still exercises the
 * kernel's tile-to-tile path (staging the next tile, crossing row and
 * lattice boundaries) that large lattices take.  Results do not depend on
 * n.  Host-side only; LBM_ERR_ARG for a NULL context or n < 0. */
int lbm_set_max_ctas(lbm_ctx *ctx, int n);

/* The hidden-layer activation of LBM_MLP_BF16 (tanh, Eq. S10 network) applied
 * element-wise, for checking its accuracy: out[k] = act(a[k]) for n FP32
 * pre-activations a (device arrays, caller-owned, asynchronous on
 * cuda_stream).  The tensor-core step evaluates some hidden units on the XU
 * and the others on the FMA pipe:
 *   path 0: the XU form, bf16 rounding then tanh.approx.bf16x2 (a bf16 value);
 *   path 1: the FMA form as the step stores it, y P(min(y^2, 1)) with
 *           y = a/4 and a degree-8 polynomial P, rounded to bf16 and clamped
 *           to [-1, 1] (a bf16 value);
 *   path 2: the FMA form before its bf16 rounding (FP32, clamped to [-1, 1]).
 * LBM_ERR_ARG for a NULL pointer, n < 0 or another path. */
int lbm_activation(const float *a, int n, int path, float *out, void *cuda_stream);

/* Compiled layout of the LBM_MLP_BF16 step kernel (no counterpart in the
 * paper; for performance accounting): *warpgroups_per_sm tiles of 128 nodes in
 * flight per SM, and *xu_pairs_per_8 -- of every 8 pairs of hidden units, how
 * many the XU evaluates (path 0 of lbm_activation; the rest use path 1).
 * Either pointer may be NULL.  Host-only, no GPU needed; returns LBM_OK. */
int lbm_mlp_bf16_layout(int *warpgroups_per_sm, int *xu_pairs_per_8);

/* Velocity loss of the current state against targets (utx, uty) [b][y][x]:
 * L = 1/(2 N B) sum |u - u_t|^2 with u = j/rho of the pre-collision
 * populations (velocity form of Eq. S13), written to loss[0] (device,
 * deterministic two-pass reduction), and, if dL_df is not NULL, its
 * gradient with respect to the pre-collision populations [b][i][y][x]. */
int lbm_velocity_loss(lbm_ctx *ctx, const float *utx, const float *uty, float *loss,
                      float *dL_df);

/* Losses on a subset S of nodes (SI section 2, "Unrolled training": the loss
 * is taken on a random subset of lattice points, |S| = 512 in the paper).
 * idx: device array of `count` node indices n = b*ny*nx + y*nx + x, each in
 * [0, batch*ny*nx); a repeated index counts once per occurrence.  An index out
 * of range adds nothing and makes the next lbm_status return LBM_ERR_ARG.
 * 1 <= count <= batch*ny*nx, else LBM_ERR_ARG before any launch.  loss[0]
 * (device float) is a deterministic two-pass FP64 reduction.  dL_df
 * (device, nullable, 9*batch*ny*nx floats) is overwritten with the gradient
 * with respect to the CURRENT pre-collision populations [b][i][y][x] (zero
 * off the entries S touches), ready for lbm_backward.
 *
 * lbm_velocity_loss_subset: velocity form,
 *   L = 1/(2|S|) sum_{n in S} |u(n) - u_t(n)|^2, u = j/rho of the pre-collision
 *   populations, targets utx, uty [b][y][x] (device).
 * lbm_population_loss_subset: Eq. S13 as printed (a plain sum),
 *   L = sum_{n in S} sum_i (g_i(n) - t_i(n))^2, g the post-collision
 *   populations of the last step (the state before streaming) and t the
 *   target post-collision populations [b][i][y][x] (device), e.g. anti-
 *   streamed filtered DNS populations (lbm_stream with dir = -1).  The
 *   gradient of g_i(n) is stored at dL/df_i(n + c_i), where g_i(n) streams to. */
int lbm_velocity_loss_subset(lbm_ctx *ctx, const int *idx, int count, const float *utx,
                             const float *uty, float *loss, float *dL_df);
int lbm_population_loss_subset(lbm_ctx *ctx, const int *idx, int count, const float *target_post,
                               float *loss, float *dL_df);

/* Streaming of a population field on the context's grid (Eq. S2), out of
 * place on the context's stream: dir = +1 streams, out_i(x) = in_i(x - c_i);
 * dir = -1 anti-streams (SI section 2, step 4: post-collision populations at
 * t from pre-collision ones at t + 1), out_i(x) = in_i(x + c_i).  in, out:
 * device [b][i][y][x], 9*batch*ny*nx floats, distinct.  The state is not
 * touched.  LBM_ERR_ARG for a null or identical pointer or another dir. */
int lbm_stream(lbm_ctx *ctx, int dir, const float *in, float *out);

/* Bytes of the workspace lbm_forward_record / lbm_backward need for an
 * n-step unroll with a checkpoint every ckpt_every steps. */
size_t lbm_record_bytes(const lbm_params *p, int n, int ckpt_every);

/* Unrolled training forward (SI section 2): advance n steps with the FP32
 * learned collision, storing the state every ckpt_every steps into `ws`
 * (device, >= lbm_record_bytes).  The start state is copied into `ws`; each
 * later checkpoint is written there by the step that produces it (no copy),
 * and the states inside the last segment are kept in the workspace's
 * recompute area, so the backward recomputes only the earlier segments.
 * The context ends at step n, as after lbm_step(n, LBM_MLP_F32). */
int lbm_forward_record(lbm_ctx *ctx, int n, int ckpt_every, const lbm_weights *w, void *ws,
                       size_t ws_bytes);

/* Hand-written adjoint of the recorded unroll.  dL_df_final is dL/d(pre-
 * collision populations) at the final time (e.g. from lbm_velocity_loss).
 * Recomputes each segment from its checkpoint, runs the per-step adjoint
 * (transpose of the pull = push; vector-Jacobian product of the learned
 * collision), and writes dL/dtheta (LBM_MLP_NPARAMS floats, packed w1, b1,
 * w2, b2, w3, b3; overwritten; deterministic) to dW and, if not NULL,
 * dL/d(pre-collision populations at the start) to dL_df0.  Uses the `ws`
 * of the matching lbm_forward_record (n and ckpt_every are remembered by the
 * context); the context's state is not changed.  The weights must be FP32
 * (dtype 0). */
int lbm_backward(lbm_ctx *ctx, const float *dL_df_final, const lbm_weights *w, void *ws,
                 size_t ws_bytes, float *dW, float *dL_df0);

/* The same unrolled training pair with the MLP on the tensor cores:
 * lbm_forward_record_bf16 advances with LBM_MLP_BF16; lbm_backward_bf16
 * recomputes segments with LBM_MLP_BF16 and runs the adjoint as tcgen05 GEMMs
 * (BF16 operands -- activations, adjoints and weights rounded to bf16 --
 * FP32 accumulation; the per-node chain rule through equilibrium,
 * projection, BGK and force in FP32), including the weight-gradient sums
 * over nodes.  Either backward may follow either record: segments are
 * recomputed with the collision the record used.  Gradients carry the bf16
 * rounding of activations and adjoints: a few per cent relative L2 of dtheta
 * for a velocity loss (whose weight-gradient sums over nodes cancel strongly),
 * against 1e-4 for the FP32 adjoint.  Same arguments and conventions as the
 * FP32 pair; lbm_backward_bf16 takes lattices of fewer than 2^31 / 9
 * population values in all (nx * ny * batch < 238,609,295) and returns
 * LBM_ERR_ARG beyond that. */
int lbm_forward_record_bf16(lbm_ctx *ctx, int n, int ckpt_every, const lbm_weights *w, void *ws,
                            size_t ws_bytes);
int lbm_backward_bf16(lbm_ctx *ctx, const float *dL_df_final, const lbm_weights *w, void *ws,
                      size_t ws_bytes, float *dW, float *dL_df0);

/* Coarse-graining filter (SI section 2, with a box average as filter phi):
 * f_coarse[b][i][J][I] = mean over the cg x cg block of the CURRENT
 * pre-collision populations of ctx_fine.  nx, ny must be multiples of cg. */
int lbm_box_filter(lbm_ctx *ctx_fine, int cg, float *f_coarse);

/* Coarse-graining by subsampling, the filter phi the paper uses (SI section
 * 2: one lattice point in every cg along each axis): f_coarse[b][i][J][I] =
 * the CURRENT pre-collision populations of ctx_fine at (x, y) = (cg I, cg J).
 * f_coarse: device, 9*batch*(ny/cg)*(nx/cg) floats.  nx, ny must be
 * multiples of cg >= 1, else LBM_ERR_ARG. */
int lbm_subsample(lbm_ctx *ctx_fine, int cg, float *f_coarse);

/* Longitudinal velocity structure functions of the current pre-collision
 * velocity (SI section 3): S[(p-1)*rmax + r-1] = < [(u(x + r e) - u(x)) . e]^p >
 * for p = 1..6, r = 1..rmax (1 <= rmax <= 65535), averaged over every node of
 * every lattice and over the two lattice directions e (periodic).  S is a
 * device array of 6*rmax doubles; deterministic.  Allocates diagnostics
 * scratch in the context on first use. */
int lbm_structure_functions(lbm_ctx *ctx, int rmax, double *S);

/* Shell-averaged kinetic energy spectrum of the current pre-collision
 * velocity (the energy spectra of the main text): E[k], k = 0..kmax,
 * E(k) = 1/2 sum over wavevectors with round(|k'|) = k of |u_hat(k')|^2 / N^2
 * (unnormalised 2D DFT, N = nx*ny, k' in grid units), averaged over the batch,
 * so that the sum over all shells is <|u|^2>/2.  E is a device array of
 * kmax+1 doubles; deterministic.  The DFT is a cuFFT call; allocates
 * diagnostics scratch and an FFT plan in the context on first use. */
int lbm_energy_spectrum(lbm_ctx *ctx, int kmax, double *E);

/* Host-buffer convenience: copy f_pre_host (pinned or pageable host memory,
 * [b][i][y][x]) in, advance n steps with `kind`, copy the final rho, ux, uy
 * to host arrays (any may be NULL).  Synchronous. */
int lbm_run_host(lbm_ctx *ctx, const float *f_pre_host, int n, lbm_collision kind,
                 const lbm_weights *w, float *rho_host, float *ux_host, float *uy_host);

/* Velocity loss without any device allocation.  The paper has no counterpart:
 * this is a service for callers that must not call cudaMalloc -- an
 * application whose device memory belongs to its own pool allocator (for
 * example a framework's caching allocator, or a service whose memory budget
 * is fixed before it starts), or a latency-critical loop where an allocation
 * or a free would synchronise the device.  Such callers cannot create a
 * context (lbm_init allocates its scratch), so this function takes the state
 * buffer directly.
 *
 * Computes exactly what lbm_velocity_loss computes, with the same kernels:
 * `state` is a device state buffer in the library's internal representation
 * ([b][i][y][x], post-collision populations minus w_i, as returned by
 * lbm_state_buffer) of a batch x ny x nx lattice; utx, uty [b][y][x]
 * targets; loss[0] receives L = 1/(2 N B) sum |u - u_t|^2 of the
 * pre-collision velocity; dL_df (nullable) receives dL/d(pre-collision
 * populations) [b][i][y][x].  All device pointers, caller-owned; the call is
 * asynchronous on `cuda_stream` (a cudaStream_t; NULL = legacy default).
 *
 * Scratch: the per-block partial sums live in one fixed array of 2^20 floats
 * (4 MiB) that the library keeps in device memory; every GPU that loads the
 * library holds it until the process exits.  Sizes needing more partial sums
 * than that -- ceil(nx / 128) * ny * batch > 1048576 -- are rejected with
 * LBM_ERR_ARG before anything is launched.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, no allocation) and caches
 * it; make that first call before any stream capture.  All calls share the
 * array, and each call overwrites the partial sums it uses, so nothing from an
 * earlier call needs clearing -- but calls that overlap on the GPU (for
 * example on two streams at once) race on the array and must be serialised by
 * the caller.  Calls no cudaMalloc, cudaFree or allocating library routine.
 * ny and batch must not exceed 65535 (they index the launch grid), else
 * LBM_ERR_ARG.
 * Returns LBM_OK, LBM_ERR_ARG (null pointer, size <= 0, or beyond the limit),
 * LBM_ERR_UNSUPPORTED (device ordinal >= 256) or LBM_ERR_CUDA. */
int lbm_velocity_loss_noalloc(const float *state, int nx, int ny, int batch, const float *utx,
                              const float *uty, float *loss, float *dL_df, void *cuda_stream);

/* Static description of an error code. */
const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
