// lbm_api.cu -- the C ABI declared in include/lbm.h: argument checking,
// the context (stream, ping-pong state buffers, small scratch), and the
// launch sequences of every entry point.  No arithmetic of the method lives
// here; it is all in the kernels.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "kernels.h"
#include "lattice.cuh"

using lbm::CollideParams;
using lbm::Grid;
using lbm::MlpF32;

struct lbm_ctx {
  lbm_params p;
  Grid g;
  float *buf[2];
  int cur;
  cudaStream_t stream;
  int device;
  int sms;
  CollideParams cp;
  // scratch (library-owned, device)
  int *d_flag;          // [0] unstable, [1] device wait timeout, [2] bad node index
  float *d_force;       // ny floats, or nullptr
  float *d_loss_part;   // lbm::loss_partials(g) doubles (float or double partials)
  float *d_dw_part;     // dw_rows * NPARAMS floats (allocated on first use)
  int dw_rows;
  // diagnostics scratch (allocated on first use)
  float *d_diag_u;      // [2B][ny][nx]
  void *d_diag_uh;      // complex [2B][ny][nx/2+1]
  double *d_diag_part;  // partial sums
  size_t diag_part_cap;
  void *fft_plan;
  unsigned wait_limit;  // polls per bounded device wait of the tensor-core kernels (0: default)
  int max_ctas;         // CTAs of the tensor-core step (0: one per SM)
  // last lbm_forward_record
  int rec_n, rec_k;
  const void *rec_ws;
  lbm_collision rec_kind;
  bool rec_last_seg;  // the recompute area of rec_ws holds the last segment's states
};

namespace {

#define CUDA_TRY(expr)                          \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return LBM_ERR_CUDA; \
  } while (0)

// Largest lattice every kernel can address: the node-per-thread kernels put
// ny and batch in gridDim.y and gridDim.z (at most 65535 each); the tiled
// tensor-core kernels count nodes of one plane (nx*ny) and 128-node tiles
// (ceil(nx/128)*ny*batch) in 32-bit integers; element offsets are 64-bit.
bool bad_params(const lbm_params *p) {
  if (!p) return true;
  if (p->nx < 1 || p->ny < 1 || p->batch < 1) return true;
  if (p->ny > 65535 || p->batch > 65535) return true;
  if ((long long)p->nx * p->ny > 0x7FFFFFFFLL) return true;
  if (((long long)p->nx + 127) / 128 * p->ny * p->batch > 0x7FFFFFFFLL) return true;
  if ((long long)p->nx * p->ny * p->batch * 9 > (1LL << 40)) return true;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return true;
  if (!(p->smag_cs >= 0.0) || !(p->smag_delta > 0.0)) return true;
  if (!std::isfinite(p->force_amp) || p->flags != 0) return true;
  return false;
}

int check_weights(lbm_collision kind, const lbm_weights *w) {
  if (kind == LBM_BGK || kind == LBM_SMAG) return LBM_OK;
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3) return LBM_ERR_ARG;
  if (w->dtype != 0 && w->dtype != 1) return LBM_ERR_ARG;
  if (kind == LBM_MLP_F32 && w->dtype != 0) return LBM_ERR_UNSUPPORTED;
  return LBM_OK;
}

MlpF32 f32_view(const lbm_weights *w) {
  MlpF32 m;
  m.w1 = static_cast<const float *>(w->w1);
  m.b1 = static_cast<const float *>(w->b1);
  m.w2 = static_cast<const float *>(w->w2);
  m.b2 = static_cast<const float *>(w->b2);
  m.w3 = static_cast<const float *>(w->w3);
  m.b3 = static_cast<const float *>(w->b3);
  return m;
}

// One step from `in` to `out` with the given collision.  `chain`: the previous
// operation on the stream is a step of the same collision issued by the same
// call (no copy or other kernel in between), so the tensor-core step may start
// its prologue while that one finishes (programmatic dependent launch).
cudaError_t one_step(lbm_ctx *c, const float *in, float *out, lbm_collision kind,
                     const lbm_weights *w, bool chain = false) {
  switch (kind) {
    case LBM_BGK: return lbm::launch_step_bgk(c->g, in, out, c->cp, c->d_flag, c->stream);
    case LBM_SMAG: return lbm::launch_step_smag(c->g, in, out, c->cp, c->d_flag, c->stream);
    case LBM_MLP_F32:
      return lbm::launch_step_mlp_f32(c->g, in, out, c->cp, f32_view(w), c->d_flag, c->stream);
    case LBM_MLP_BF16: {
      const void *wp[6] = {w->w1, w->b1, w->w2, w->b2, w->w3, w->b3};
      return lbm::launch_step_mlp_bf16(c->g, in, out, c->cp, wp, w->dtype, c->d_flag,
                                       c->d_flag + 1, c->stream, c->wait_limit, c->max_ctas,
                                       chain);
    }
  }
  return cudaErrorInvalidValue;
}

int ensure_dw_partials(lbm_ctx *c) {
  if (c->d_dw_part) return LBM_OK;
  const int a = lbm::adjoint_blocks(c->g, c->sms), b = lbm::adjoint_tc_rows(c->g, c->sms);
  c->dw_rows = a > b ? a : b;  // capacity; each adjoint uses its own row count
  CUDA_TRY(cudaMalloc(&c->d_dw_part, (size_t)c->dw_rows * lbm::NPARAMS * sizeof(float)));
  return LBM_OK;
}

int ensure_diag(lbm_ctx *c, size_t part_doubles) {
  if (!c->d_diag_u) {
    CUDA_TRY(cudaMalloc(&c->d_diag_u, sizeof(float) * 2 * c->g.nodes()));
    CUDA_TRY(cudaMalloc(&c->d_diag_uh, sizeof(float) * 2 * 2 * (size_t)c->g.batch * c->g.ny *
                                           (c->g.nx / 2 + 1)));
  }
  if (part_doubles > c->diag_part_cap) {
    cudaFree(c->d_diag_part);
    c->d_diag_part = nullptr;
    c->diag_part_cap = 0;
    CUDA_TRY(cudaMalloc(&c->d_diag_part, sizeof(double) * part_doubles));
    c->diag_part_cap = part_doubles;
  }
  return LBM_OK;
}

size_t state_bytes(const lbm_params *p) {
  return (size_t)9 * p->nx * p->ny * p->batch * sizeof(float);
}

int n_checkpoints(int n, int k) { return n == 0 ? 1 : (n + k - 1) / k; }

}  // namespace

extern "C" {

const char *lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_UNSUPPORTED: return "not supported by this library";
    case LBM_ERR_UNSTABLE: return "unstable: |u| >= 0.4 or non-finite velocity";
    case LBM_ERR_TIMEOUT: return "a bounded device wait gave up";
  }
  return "unknown error";
}

int lbm_init(lbm_ctx **out, const lbm_params *p, float *f_buf0, float *f_buf1,
             void *cuda_stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (bad_params(p) || !f_buf0 || !f_buf1 || f_buf0 == f_buf1) return LBM_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(f_buf0) | reinterpret_cast<uintptr_t>(f_buf1)) & 15)
    return LBM_ERR_ARG;  // 16-byte alignment for the vector loads
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_ARG;
  c->p = *p;
  c->g = Grid{p->nx, p->ny, p->batch};
  c->buf[0] = f_buf0;
  c->buf[1] = f_buf1;
  c->cur = 0;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return LBM_ERR_CUDA;
  }
  c->cp.tau = (float)p->tau;
  c->cp.omega = (float)(1.0 / p->tau);
  c->cp.tau0_sq = (float)(p->tau * p->tau);
  c->cp.smag_c18 = (float)(18.0 * (p->smag_cs * p->smag_delta) * (p->smag_cs * p->smag_delta));
  c->cp.force = nullptr;
  int rc = LBM_OK;
  if (cudaMalloc(&c->d_flag, 3 * sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_flag, 0, 3 * sizeof(int)) != cudaSuccess)
    rc = LBM_ERR_CUDA;
  if (rc == LBM_OK && p->force_amp != 0.0) {
    // F_x(y) = F0 sin(2 pi m y / ny), evaluated in double on the host
    float *h = static_cast<float *>(std::malloc(sizeof(float) * p->ny));
    if (!h) rc = LBM_ERR_ARG;
    for (int y = 0; rc == LBM_OK && y < p->ny; ++y)
      h[y] = (float)(p->force_amp * std::sin(2.0 * M_PI * (double)p->force_mode * y / p->ny));
    if (rc == LBM_OK && (cudaMalloc(&c->d_force, sizeof(float) * p->ny) != cudaSuccess ||
                         cudaMemcpy(c->d_force, h, sizeof(float) * p->ny,
                                    cudaMemcpyHostToDevice) != cudaSuccess))
      rc = LBM_ERR_CUDA;
    std::free(h);
    c->cp.force = c->d_force;
  }
  if (rc == LBM_OK &&
      cudaMalloc(&c->d_loss_part, sizeof(double) * lbm::loss_partials(c->g)) != cudaSuccess)
    rc = LBM_ERR_CUDA;
  if (rc != LBM_OK) {
    lbm_destroy(c);
    return rc;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  cudaFree(c->d_flag);
  cudaFree(c->d_force);
  cudaFree(c->d_loss_part);
  cudaFree(c->d_dw_part);
  cudaFree(c->d_diag_u);
  cudaFree(c->d_diag_uh);
  cudaFree(c->d_diag_part);
  lbm::destroy_spectrum_plan(c->fft_plan);
  delete c;
}

float *lbm_state_buffer(lbm_ctx *c) { return c ? c->buf[c->cur] : nullptr; }

int lbm_set_state(lbm_ctx *c, const float *f_pre) {
  if (!c || !f_pre) return LBM_ERR_ARG;
  if (f_pre == c->buf[c->cur]) return LBM_ERR_ARG;  // the anti-stream needs a separate source
  CUDA_TRY(lbm::launch_set_state(c->g, f_pre, c->buf[c->cur], c->stream));
  return LBM_OK;
}

int lbm_get_state(lbm_ctx *c, float *f_pre) {
  if (!c || !f_pre || f_pre == c->buf[c->cur]) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_get_state(c->g, c->buf[c->cur], f_pre, c->stream));
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_ctx *c, const float *rho, const float *ux, const float *uy) {
  if (!c || !rho || !ux || !uy) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_init_equilibrium(c->g, rho, ux, uy, c->buf[c->cur], c->stream));
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n, lbm_collision kind, const lbm_weights *w) {
  if (!c || n < 0) return LBM_ERR_ARG;
  if (kind < LBM_BGK || kind > LBM_MLP_F32) return LBM_ERR_ARG;
  const int wc = check_weights(kind, w);
  if (wc != LBM_OK) return wc;
  for (int s = 0; s < n; ++s) {
    CUDA_TRY(one_step(c, c->buf[c->cur], c->buf[c->cur ^ 1], kind, w, s > 0));
    c->cur ^= 1;
  }
  return LBM_OK;
}

int lbm_moments(lbm_ctx *c, float *rho, float *ux, float *uy) {
  if (!c) return LBM_ERR_ARG;
  if (!rho && !ux && !uy) return LBM_OK;
  CUDA_TRY(lbm::launch_moments(c->g, c->buf[c->cur], rho, ux, uy, c->stream));
  return LBM_OK;
}

int lbm_status(lbm_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  int h[3] = {0, 0, 0};
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpy(h, c->d_flag, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[1]) return LBM_ERR_TIMEOUT;
  if (h[2]) return LBM_ERR_ARG;
  if (h[0]) return LBM_ERR_UNSTABLE;
  return LBM_OK;
}

int lbm_clear_status(lbm_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, 3 * sizeof(int), c->stream));
  return LBM_OK;
}

int lbm_mlp_bf16_layout(int *warpgroups_per_sm, int *xu_pairs_per_8) {
  lbm::mlp_bf16_layout(warpgroups_per_sm, xu_pairs_per_8);
  return LBM_OK;
}

int lbm_activation(const float *a, int n, int path, float *out, void *cuda_stream) {
  if (!a || !out || n < 0 || path < 0 || path > 2) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_activation(a, n, path, out, static_cast<cudaStream_t>(cuda_stream)));
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx *c, unsigned polls) {
  if (!c) return LBM_ERR_ARG;
  c->wait_limit = polls;
  return LBM_OK;
}

int lbm_set_max_ctas(lbm_ctx *c, int n) {
  if (!c || n < 0) return LBM_ERR_ARG;
  c->max_ctas = n;
  return LBM_OK;
}

int lbm_velocity_loss(lbm_ctx *c, const float *utx, const float *uty, float *loss,
                      float *dL_df) {
  if (!c || !utx || !uty || !loss) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_velocity_loss(c->g, c->buf[c->cur], utx, uty, c->d_loss_part, loss, dL_df,
                                     c->stream));
  return LBM_OK;
}

int lbm_velocity_loss_subset(lbm_ctx *c, const int *idx, int count, const float *utx,
                             const float *uty, float *loss, float *dL_df) {
  if (!c || !idx || !utx || !uty || !loss) return LBM_ERR_ARG;
  if (count < 1 || (size_t)count > c->g.nodes()) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_velocity_loss_subset(c->g, c->buf[c->cur], idx, count, utx, uty,
                                            reinterpret_cast<double *>(c->d_loss_part), loss,
                                            dL_df, c->d_flag + 2, c->stream));
  return LBM_OK;
}

int lbm_population_loss_subset(lbm_ctx *c, const int *idx, int count, const float *target_post,
                               float *loss, float *dL_df) {
  if (!c || !idx || !target_post || !loss) return LBM_ERR_ARG;
  if (count < 1 || (size_t)count > c->g.nodes()) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_population_loss_subset(c->g, c->buf[c->cur], idx, count, target_post,
                                              reinterpret_cast<double *>(c->d_loss_part), loss,
                                              dL_df, c->d_flag + 2, c->stream));
  return LBM_OK;
}

int lbm_stream(lbm_ctx *c, int dir, const float *in, float *out) {
  if (!c || !in || !out || in == out || (dir != 1 && dir != -1)) return LBM_ERR_ARG;
  // dir +1 streams (out_i(x) = in_i(x - c_i)), the launcher's pull; -1 anti-streams
  if (dir == 1)
    CUDA_TRY(lbm::launch_pull(c->g, in, out, c->stream));
  else
    CUDA_TRY(lbm::launch_push(c->g, in, out, c->stream));
  return LBM_OK;
}

size_t lbm_record_bytes(const lbm_params *p, int n, int k) {
  if (bad_params(p) || n < 0 || k < 1) return 0;
  // checkpoints + (k - 1) recomputed states of one segment + 2 adjoint buffers
  const size_t states = (size_t)n_checkpoints(n, k) + (size_t)(k - 1) + 2;
  return states * state_bytes(p);
}

}  // extern "C"

static int forward_record(lbm_ctx *c, lbm_collision kind, int n, int k, const lbm_weights *w,
                          void *ws, size_t ws_bytes) {
  if (!c || n < 0 || k < 1 || !ws) return LBM_ERR_ARG;
  if (!w || check_weights(LBM_MLP_F32, w) != LBM_OK) return LBM_ERR_ARG;
  if (ws_bytes < lbm_record_bytes(&c->p, n, k)) return LBM_ERR_ARG;
  const size_t sb = state_bytes(&c->p);
  char *base = static_cast<char *>(ws);
  // Checkpoint 0 is a copy of the current state.  Every later checkpoint
  // g^{jk} (jk < n) is written there by the step that produces it, and the
  // next step reads it from there, so the record costs one copy, not n/k.
  // The states inside the last segment, g^{s0+1} .. g^{n-1}, go where the
  // backward would recompute them (the workspace's k - 1 recompute states),
  // so the backward starts without a recompute.  The other steps alternate
  // between the two state buffers, and the last one (g^n is never stored in
  // the workspace) ends in a state buffer.
  const int last_s0 = n > 0 ? ((n - 1) / k) * k : 0;
  float *seg = reinterpret_cast<float *>(base + (size_t)n_checkpoints(n, k) * sb);
  const size_t sf = sb / sizeof(float);
  c->rec_last_seg = false;
  CUDA_TRY(cudaMemcpyAsync(base, c->buf[c->cur], sb, cudaMemcpyDeviceToDevice, c->stream));
  const float *in = c->buf[c->cur];
  for (int s = 0; s < n; ++s) {
    const int t = s + 1;  // the state this step produces
    float *out;
    bool to_buf = false;
    if (t % k == 0 && t < n)
      out = reinterpret_cast<float *>(base + (size_t)(t / k) * sb);
    else if (t > last_s0 && t < n)
      out = seg + (size_t)(t - last_s0 - 1) * sf;
    else
      out = c->buf[c->cur ^ 1], to_buf = true;
    CUDA_TRY(one_step(c, in, out, kind, w, s > 0));
    if (to_buf) c->cur ^= 1;
    in = out;
  }
  c->rec_n = n;
  c->rec_k = k;
  c->rec_ws = ws;
  c->rec_kind = kind;
  c->rec_last_seg = n > 0;
  return LBM_OK;
}

extern "C" int lbm_forward_record(lbm_ctx *c, int n, int k, const lbm_weights *w, void *ws,
                                  size_t ws_bytes) {
  return forward_record(c, LBM_MLP_F32, n, k, w, ws, ws_bytes);
}

extern "C" int lbm_forward_record_bf16(lbm_ctx *c, int n, int k, const lbm_weights *w, void *ws,
                                       size_t ws_bytes) {
  return forward_record(c, LBM_MLP_BF16, n, k, w, ws, ws_bytes);
}

static int backward(lbm_ctx *c, bool tc, const float *dL_df_final, const lbm_weights *w, void *ws,
                    size_t ws_bytes, float *dW, float *dL_df0) {
  if (!c || !dL_df_final || !ws || !dW) return LBM_ERR_ARG;
  if (!w || check_weights(LBM_MLP_F32, w) != LBM_OK) return LBM_ERR_ARG;
  if (ws != c->rec_ws) return LBM_ERR_ARG;  // needs the workspace of the last record
  // the tensor-core adjoint's launcher takes fewer than 2^31 population values
  if (tc && (long long)c->g.nodes() * 9 >= (1LL << 31)) return LBM_ERR_ARG;
  // segments are recomputed with the collision the record used
  const lbm_collision kind = c->rec_kind;
  const int n = c->rec_n, k = c->rec_k;
  if (ws_bytes < lbm_record_bytes(&c->p, n, k)) return LBM_ERR_ARG;
  int rc = ensure_dw_partials(c);
  if (rc != LBM_OK) return rc;
  const int rows = tc ? lbm::adjoint_tc_rows(c->g, c->sms) : lbm::adjoint_blocks(c->g, c->sms);
  const size_t sb = state_bytes(&c->p);
  char *base = static_cast<char *>(ws);
  const int nck = n_checkpoints(n, k);
  float *seg = reinterpret_cast<float *>(base + (size_t)nck * sb);  // k - 1 states
  float *lam[2] = {reinterpret_cast<float *>(base + (size_t)(nck + k - 1) * sb),
                   reinterpret_cast<float *>(base + (size_t)(nck + k) * sb)};
  const size_t sf = sb / sizeof(float);
  const MlpF32 wf = f32_view(w);
  // lam = dL/d(stored state g^n): the transpose of the final pull is a push
  CUDA_TRY(lbm::launch_push(c->g, dL_df_final, lam[0], c->stream));
  int cur = 0;
  bool first = true;
  const int last_s0 = n > 0 ? ((n - 1) / k) * k : 0;
  for (int s0 = last_s0; n > 0 && s0 >= 0; s0 -= k) {
    const float *ck = reinterpret_cast<const float *>(base + (size_t)(s0 / k) * sb);
    const int len = (s0 + k <= n) ? k : n - s0;
    // g^{s0+1} .. g^{s0+len-1} in seg[0 .. len-2]: left there by the record
    // for the last segment (until a recompute of another segment overwrites
    // them), recomputed from the checkpoint otherwise
    if (!(s0 == last_s0 && c->rec_last_seg) && len > 1) {
      for (int j = 1; j < len; ++j) {
        const float *in = j == 1 ? ck : seg + (size_t)(j - 2) * sf;
        CUDA_TRY(one_step(c, in, seg + (size_t)(j - 1) * sf, kind, w, j > 1));
      }
      c->rec_last_seg = s0 == last_s0;
    }
    for (int j = len - 1; j >= 0; --j) {
      const float *gs = j == 0 ? ck : seg + (size_t)(j - 1) * sf;
      if (tc)
        CUDA_TRY(lbm::launch_adjoint_tc(c->g, gs, lam[cur], lam[cur ^ 1], c->cp, wf,
                                        c->d_dw_part, rows, first ? 0 : 1, c->d_flag + 1,
                                        c->stream));
      else
        CUDA_TRY(lbm::launch_adjoint_step(c->g, gs, lam[cur], lam[cur ^ 1], c->cp, wf,
                                          c->d_dw_part, rows, first ? 0 : 1, c->stream));
      first = false;
      cur ^= 1;
    }
  }
  if (first) {
    CUDA_TRY(cudaMemsetAsync(dW, 0, sizeof(float) * lbm::NPARAMS, c->stream));
  } else {
    CUDA_TRY(lbm::launch_reduce_dw(c->d_dw_part, rows, dW, c->stream));
  }
  // dL/df_pre(0) = pull(lam^0): g^0 was the push of f_pre(0)
  if (dL_df0) CUDA_TRY(lbm::launch_pull(c->g, lam[cur], dL_df0, c->stream));
  return LBM_OK;
}

extern "C" int lbm_backward(lbm_ctx *c, const float *dL_df_final, const lbm_weights *w,
                            void *ws, size_t ws_bytes, float *dW, float *dL_df0) {
  return backward(c, false, dL_df_final, w, ws, ws_bytes, dW, dL_df0);
}

extern "C" int lbm_backward_bf16(lbm_ctx *c, const float *dL_df_final, const lbm_weights *w,
                                 void *ws, size_t ws_bytes, float *dW, float *dL_df0) {
  return backward(c, true, dL_df_final, w, ws, ws_bytes, dW, dL_df0);
}

extern "C" {

int lbm_structure_functions(lbm_ctx *c, int rmax, double *S) {
  if (!c || !S || rmax < 1 || rmax > 65535) return LBM_ERR_ARG;
  const int rc = ensure_diag(c, lbm::structure_partials_doubles(c->g, rmax));
  if (rc != LBM_OK) return rc;
  float *ux = c->d_diag_u, *uy = c->d_diag_u + c->g.nodes();
  CUDA_TRY(lbm::launch_moments(c->g, c->buf[c->cur], nullptr, ux, uy, c->stream));
  CUDA_TRY(lbm::launch_structure_functions(c->g, ux, uy, rmax, c->d_diag_part, S, c->stream));
  return LBM_OK;
}

int lbm_energy_spectrum(lbm_ctx *c, int kmax, double *E) {
  if (!c || !E || kmax < 0 || kmax > (1 << 24)) return LBM_ERR_ARG;
  const int rc = ensure_diag(c, lbm::spectrum_rowpart_doubles(c->g, kmax));
  if (rc != LBM_OK) return rc;
  float *ux = c->d_diag_u, *uy = c->d_diag_u + c->g.nodes();
  CUDA_TRY(lbm::launch_moments(c->g, c->buf[c->cur], nullptr, ux, uy, c->stream));
  CUDA_TRY(lbm::launch_energy_spectrum(c->g, c->d_diag_u, c->d_diag_uh, &c->fft_plan, kmax,
                                       c->d_diag_part, E, c->stream));
  return LBM_OK;
}

int lbm_box_filter(lbm_ctx *c, int cg, float *f_coarse) {
  if (!c || !f_coarse || cg < 1) return LBM_ERR_ARG;
  if (c->g.nx % cg || c->g.ny % cg) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_box_filter(c->g, c->buf[c->cur], cg, f_coarse, c->stream));
  return LBM_OK;
}

int lbm_subsample(lbm_ctx *c, int cg, float *f_coarse) {
  if (!c || !f_coarse || cg < 1) return LBM_ERR_ARG;
  if (c->g.nx % cg || c->g.ny % cg) return LBM_ERR_ARG;
  CUDA_TRY(lbm::launch_subsample(c->g, c->buf[c->cur], cg, f_coarse, c->stream));
  return LBM_OK;
}

int lbm_run_host(lbm_ctx *c, const float *f_pre_host, int n, lbm_collision kind,
                 const lbm_weights *w, float *rho_host, float *ux_host, float *uy_host) {
  if (!c || !f_pre_host || n < 0) return LBM_ERR_ARG;
  if (kind < LBM_BGK || kind > LBM_MLP_F32) return LBM_ERR_ARG;
  const int wc = check_weights(kind, w);
  if (wc != LBM_OK) return wc;
  const size_t sb = state_bytes(&c->p);
  // the non-current buffer stages the input, then the output fields
  float *stage = c->buf[c->cur ^ 1];
  CUDA_TRY(cudaMemcpyAsync(stage, f_pre_host, sb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(lbm::launch_set_state(c->g, stage, c->buf[c->cur], c->stream));
  int rc = lbm_step(c, n, kind, w);
  if (rc != LBM_OK) return rc;
  const size_t nn = c->g.nodes();
  float *out = c->buf[c->cur ^ 1];
  CUDA_TRY(lbm::launch_moments(c->g, c->buf[c->cur], out, out + nn, out + 2 * nn, c->stream));
  if (rho_host)
    CUDA_TRY(cudaMemcpyAsync(rho_host, out, nn * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (ux_host)
    CUDA_TRY(cudaMemcpyAsync(ux_host, out + nn, nn * sizeof(float), cudaMemcpyDeviceToHost,
                             c->stream));
  if (uy_host)
    CUDA_TRY(cudaMemcpyAsync(uy_host, out + 2 * nn, nn * sizeof(float), cudaMemcpyDeviceToHost,
                             c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

}  // extern "C"
