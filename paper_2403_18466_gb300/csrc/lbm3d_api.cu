// lbm3d_api.cu -- the C ABI declared in include/lbm3d.h (the paper's D3Q19
// setting): argument checking, the context (stream, ping-pong buffers, status
// flag, force tables) and the launch sequences.  No arithmetic of the method
// lives here; it is all in the kernels.
#include <cmath>
#include <new>
#include <vector>

#include "../../include/lbm3d.h"
#include "d3q19.cuh"
#include "kernels3d.h"

using lbm::d3::Collide3;
using lbm::d3::Grid3;
using lbm::d3::Mlp3;

struct lbm3d_ctx {
  lbm3d_params p;
  Grid3 g;
  float *buf[2];
  int cur;
  cudaStream_t stream;
  Collide3 cp;
  int *d_flag;     // [0] unstable, [1] device wait timeout
  float *d_force;  // ny + nz + nx floats (F_x(y), F_y(z), F_z(x)), or nullptr
  void *d_wtc;     // BF16 operand tiles of the tensor-core collision (first use)
  int sms;
};

namespace {

#define CUDA_TRY(expr)                          \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return LBM_ERR_CUDA; \
  } while (0)

bool bad_params(const lbm3d_params *p) {
  if (!p) return true;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->batch < 1) return true;
  if (p->ny > 65535 || (long long)p->nz * p->batch > 65535) return true;
  if ((long long)p->nx * p->ny * p->nz * p->batch * 19 > (1LL << 40)) return true;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return true;
  if (!(p->smag_cs >= 0.0) || !(p->smag_delta > 0.0)) return true;
  if (!std::isfinite(p->force_amp) || p->flags != 0) return true;
  return false;
}

int check_weights(lbm_collision kind, const lbm3d_weights *w) {
  if (kind == LBM_BGK || kind == LBM_SMAG) return LBM_OK;
  if (kind != LBM_MLP_F32 && kind != LBM_MLP_BF16) return LBM_ERR_ARG;
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || !w->w4 || !w->b4)
    return LBM_ERR_ARG;
  if (w->dtype != 0) return LBM_ERR_UNSUPPORTED;
  return LBM_OK;
}

Mlp3 f32_view(const lbm3d_weights *w) {
  Mlp3 m;
  m.w1 = static_cast<const float *>(w->w1);
  m.b1 = static_cast<const float *>(w->b1);
  m.w2 = static_cast<const float *>(w->w2);
  m.b2 = static_cast<const float *>(w->b2);
  m.w3 = static_cast<const float *>(w->w3);
  m.b3 = static_cast<const float *>(w->b3);
  m.w4 = static_cast<const float *>(w->w4);
  m.b4 = static_cast<const float *>(w->b4);
  return m;
}

}  // namespace

extern "C" {

size_t lbm3d_mlp_nparams(void) { return (size_t)lbm::d3::NPARAMS; }

void lbm3d_lattice(int *cx, int *cy, int *cz, float *w) {
  for (int i = 0; i < lbm::d3::Q; ++i) {
    if (cx) cx[i] = lbm::d3::cx(i);
    if (cy) cy[i] = lbm::d3::cy(i);
    if (cz) cz[i] = lbm::d3::cz(i);
    if (w) w[i] = lbm::d3::wf(i);
  }
}

int lbm3d_init(lbm3d_ctx **out, const lbm3d_params *p, float *b0, float *b1, void *stream) {
  if (!out || bad_params(p) || !b0 || !b1 || b0 == b1) return LBM_ERR_ARG;
  *out = nullptr;
  lbm3d_ctx *c = new (std::nothrow) lbm3d_ctx();
  if (!c) return LBM_ERR_CUDA;
  c->p = *p;
  c->g = Grid3{p->nx, p->ny, p->nz, p->batch};
  c->buf[0] = b0;
  c->buf[1] = b1;
  c->cur = 0;
  c->stream = static_cast<cudaStream_t>(stream);
  c->cp.tau = (float)p->tau;
  c->cp.omega = (float)(1.0 / p->tau);
  c->cp.tau0_sq = (float)(p->tau * p->tau);
  c->cp.smag_c18 = (float)(18.0 * (p->smag_cs * p->smag_delta) * (p->smag_cs * p->smag_delta));
  c->cp.fx_y = c->cp.fy_z = c->cp.fz_x = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return LBM_ERR_CUDA;
  }
  if (cudaMalloc(&c->d_flag, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_flag, 0, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(c->d_flag);
    delete c;
    return LBM_ERR_CUDA;
  }
  if (p->force_amp != 0.0) {
    // sine tables in FP64 on the host, one per axis
    std::vector<float> h((size_t)p->ny + p->nz + p->nx);
    const double k = 2.0 * M_PI * (double)p->force_mode;
    for (int y = 0; y < p->ny; ++y) h[y] = (float)(p->force_amp * std::sin(k * y / p->ny));
    for (int z = 0; z < p->nz; ++z)
      h[(size_t)p->ny + z] = (float)(p->force_amp * std::sin(k * z / p->nz));
    for (int x = 0; x < p->nx; ++x)
      h[(size_t)p->ny + p->nz + x] = (float)(p->force_amp * std::sin(k * x / p->nx));
    if (cudaMalloc(&c->d_force, sizeof(float) * h.size()) != cudaSuccess ||
        cudaMemcpy(c->d_force, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaFree(c->d_force);
      cudaFree(c->d_flag);
      delete c;
      return LBM_ERR_CUDA;
    }
    c->cp.fx_y = c->d_force;
    c->cp.fy_z = c->d_force + p->ny;
    c->cp.fz_x = c->d_force + p->ny + p->nz;
  }
  *out = c;
  return LBM_OK;
}

void lbm3d_destroy(lbm3d_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_flag);
  cudaFree(c->d_force);
  cudaFree(c->d_wtc);
  delete c;
}

int lbm3d_set_state(lbm3d_ctx *c, const float *f_pre) {
  if (!c || !f_pre) return LBM_ERR_ARG;
  CUDA_TRY(lbm::d3::launch_set_state(c->g, f_pre, c->buf[c->cur], c->stream));
  return LBM_OK;
}

int lbm3d_get_state(lbm3d_ctx *c, float *f_pre) {
  if (!c || !f_pre) return LBM_ERR_ARG;
  CUDA_TRY(lbm::d3::launch_get_state(c->g, c->buf[c->cur], f_pre, c->stream));
  return LBM_OK;
}

int lbm3d_init_equilibrium(lbm3d_ctx *c, const float *rho, const float *u) {
  if (!c || !rho || !u) return LBM_ERR_ARG;
  CUDA_TRY(lbm::d3::launch_init_equilibrium(c->g, rho, u, c->buf[c->cur], c->stream));
  return LBM_OK;
}

int lbm3d_step(lbm3d_ctx *c, int n, lbm_collision kind, const lbm3d_weights *w) {
  if (!c || n < 0) return LBM_ERR_ARG;
  const int wc = check_weights(kind, w);
  if (wc != LBM_OK) return wc;
  if (kind == LBM_MLP_BF16 && n > 0) {
    if (!c->d_wtc) CUDA_TRY(cudaMalloc(&c->d_wtc, lbm::d3::mlp_tc_weight_bytes()));
    CUDA_TRY(lbm::d3::launch_prepare_weights_tc(f32_view(w), c->d_wtc, c->stream));
  }
  for (int s = 0; s < n; ++s) {
    const float *in = c->buf[c->cur];
    float *out = c->buf[c->cur ^ 1];
    if (kind == LBM_MLP_BF16)
      CUDA_TRY(lbm::d3::launch_step_mlp_tc(c->g, in, out, c->cp, c->d_wtc, c->sms, c->d_flag,
                                           c->d_flag + 1, c->stream));
    else if (kind == LBM_MLP_F32)
      CUDA_TRY(lbm::d3::launch_step_mlp_f32(c->g, in, out, c->cp, f32_view(w), c->d_flag,
                                            c->stream));
    else
      CUDA_TRY(lbm::d3::launch_step(c->g, in, out, c->cp, kind == LBM_SMAG ? 1 : 0, c->d_flag,
                                    c->stream));
    c->cur ^= 1;
  }
  return LBM_OK;
}

int lbm3d_moments(lbm3d_ctx *c, float *rho, float *u) {
  if (!c) return LBM_ERR_ARG;
  CUDA_TRY(lbm::d3::launch_moments(c->g, c->buf[c->cur], rho, u, c->stream));
  return LBM_OK;
}

float *lbm3d_state_buffer(lbm3d_ctx *c) { return c ? c->buf[c->cur] : nullptr; }

int lbm3d_status(lbm3d_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  int h[2] = {0, 0};
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpy(h, c->d_flag, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[1]) return LBM_ERR_TIMEOUT;
  if (h[0]) return LBM_ERR_UNSTABLE;
  return LBM_OK;
}

int lbm3d_clear_status(lbm3d_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, 2 * sizeof(int), c->stream));
  return LBM_OK;
}

}  // extern "C"
