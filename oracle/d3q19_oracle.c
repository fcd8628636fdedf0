/*
 * d3q19_oracle.c -- plain, slow FP64 CPU oracle of the paper's own 3D setting:
 * the D3Q19 lattice-Boltzmann step (stream, moments, equilibrium, BGK,
 * Smagorinsky-BGK, EDM forcing with the paper's three-component sine force)
 * and the learned collision with the paper's network (19 -> 300 -> 300 -> 100
 * -> 19, LeakyReLU) and its conservation layer with kappa denominators 19 and 10.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path calls this file; it
 * shares no code, header or table with the CUDA path: the stencil below is its
 * own copy of the paper's D3Q19 table (SI, "D3Q19 velocity stencil").
 *
 * Conventions
 *   - populations are SoA, index [b][i][z][y][x], x fastest;
 *   - the stored state of a run is the POST-collision populations g; the
 *     pre-collision populations of the next step are f_i(x) = g_i(x - c_i);
 *   - Delta t = Delta x = 1.
 *
 * Parity status (pins in tests/test_oracle_d3q19.py): every function pinned.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The paper's D3Q19 stencil, in the paper's index order. */
static const int O3_CX[19] = {0, -1, 0, 0, 0, 0, 1, -1, -1, -1, -1, 0, 0, 0, 0, 1, 1, 1, 1};
static const int O3_CY[19] = {0, 0, -1, 0, 0, 1, 0, -1, 0, 0, 1, -1, -1, 1, 1, -1, 0, 0, 1};
static const int O3_CZ[19] = {0, 0, 0, -1, 1, 0, 0, 0, -1, 1, 0, -1, 1, -1, 1, 0, -1, 1, 0};
static double o3_w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static const double O3_CS2 = 1.0 / 3.0;

enum { O3_BGK = 0, O3_SMAG = 1, O3_MLP = 2 };

typedef struct {
  double tau;         /* relaxation time (Eq. S3) */
  double smag_cs;     /* Smagorinsky constant */
  double smag_delta;  /* filter width, lattice units */
  double force_amp;   /* F of the sine forcing */
  int force_mode;     /* m: F_x(y) = F sin(2 pi m y / ny), F_y(z), F_z(x) alike */
  int h1, h2, h3;     /* hidden widths (the paper: 300, 300, 100) */
  double leaky_slope; /* LeakyReLU negative slope */
} o3_params;

static inline size_t idx5(int b, int i, int z, int y, int x, int nz, int ny, int nx) {
  return ((((size_t)b * 19 + i) * nz + z) * ny + y) * nx + x;
}
static inline int wrap3(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

void o3_lattice(int *cx, int *cy, int *cz, double *w) {
  for (int i = 0; i < 19; ++i) {
    cx[i] = O3_CX[i];
    cy[i] = O3_CY[i];
    cz[i] = O3_CZ[i];
    w[i] = o3_w(i);
  }
}

/* Second-order equilibrium (Eq. S4) on D3Q19. */
void o3_feq(double rho, double ux, double uy, double uz, double *feq) {
  const double usq = ux * ux + uy * uy + uz * uz;
  for (int i = 0; i < 19; ++i) {
    const double cu = O3_CX[i] * ux + O3_CY[i] * uy + O3_CZ[i] * uz;
    feq[i] = o3_w(i) * rho *
             (1.0 + cu / O3_CS2 + (cu * cu - O3_CS2 * usq) / (2.0 * O3_CS2 * O3_CS2));
  }
}

static void o3_node_moments(const double *f, double *rho, double *u) {
  double r = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 19; ++i) {
    r += f[i];
    j[0] += f[i] * O3_CX[i];
    j[1] += f[i] * O3_CY[i];
    j[2] += f[i] * O3_CZ[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* Streaming (pull) f_i(x) = g_i(x - c_i), periodic (Eq. S2). */
void o3_stream_pull(int B, int nz, int ny, int nx, const double *g, double *f) {
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 19; ++i)
#pragma omp parallel for
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x)
            f[idx5(b, i, z, y, x, nz, ny, nx)] =
                g[idx5(b, i, wrap3(z - O3_CZ[i], nz), wrap3(y - O3_CY[i], ny),
                       wrap3(x - O3_CX[i], nx), nz, ny, nx)];
}

/* Anti-streaming g_i(x) = f_i(x + c_i), the inverse of the pull. */
void o3_stream_push(int B, int nz, int ny, int nx, const double *f, double *g) {
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 19; ++i)
#pragma omp parallel for
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x)
            g[idx5(b, i, z, y, x, nz, ny, nx)] =
                f[idx5(b, i, wrap3(z + O3_CZ[i], nz), wrap3(y + O3_CY[i], ny),
                       wrap3(x + O3_CX[i], nx), nz, ny, nx)];
}

/* rho and u = j / rho per node; u is [B][3][nz][ny][nx]. */
void o3_moments(int B, int nz, int ny, int nx, const double *f, double *rho, double *u) {
  const size_t N = (size_t)nz * ny * nx;
  for (int b = 0; b < B; ++b)
#pragma omp parallel for
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double fn[19], r, v[3];
          for (int i = 0; i < 19; ++i) fn[i] = f[idx5(b, i, z, y, x, nz, ny, nx)];
          o3_node_moments(fn, &r, v);
          const size_t n = ((size_t)z * ny + y) * nx + x;
          rho[(size_t)b * N + n] = r;
          for (int a = 0; a < 3; ++a) u[((size_t)b * 3 + a) * N + n] = v[a];
        }
}

/* The paper's forcing of the 3D DNS:
 * F_x(y) = F sin(2 pi m y / ny), F_y(z) = F sin(2 pi m z / nz), F_z(x) = F sin(2 pi m x / nx). */
void o3_force(const o3_params *p, int z, int y, int x, int nz, int ny, int nx, double *F) {
  F[0] = F[1] = F[2] = 0.0;
  if (p->force_amp == 0.0) return;
  const double k = 2.0 * M_PI * (double)p->force_mode;
  F[0] = p->force_amp * sin(k * (double)y / (double)ny);
  F[1] = p->force_amp * sin(k * (double)z / (double)nz);
  F[2] = p->force_amp * sin(k * (double)x / (double)nx);
}

/* Exact Difference Method forcing (Eq. S5): feq(rho, u + F/rho) - feq(rho, u). */
void o3_edm_force(double rho, const double *u, const double *F, double *fext) {
  double a[19], s[19];
  o3_feq(rho, u[0], u[1], u[2], a);
  o3_feq(rho, u[0] + F[0] / rho, u[1] + F[1] / rho, u[2] + F[2] / rho, s);
  for (int i = 0; i < 19; ++i) fext[i] = s[i] - a[i];
}

/* Smagorinsky relaxation time (SI section 1), the same closed form as in 2D:
 * tau_eff = (tau0 + sqrt(tau0^2 + 18 (C_s Delta)^2 Q / rho)) / 2 with
 * Q = sqrt(2 Pi:Pi), Pi_ab = sum_i c_ia c_ib (f_i - feq_i). */
double o3_smag_tau_eff(const double *f, double tau0, double cs, double delta) {
  double rho, u[3], feq[19];
  o3_node_moments(f, &rho, u);
  o3_feq(rho, u[0], u[1], u[2], feq);
  double P[3][3] = {{0}};
  for (int i = 0; i < 19; ++i) {
    const double d = f[i] - feq[i];
    const int c[3] = {O3_CX[i], O3_CY[i], O3_CZ[i]};
    for (int a = 0; a < 3; ++a)
      for (int bb = 0; bb < 3; ++bb) P[a][bb] += c[a] * c[bb] * d;
  }
  double pp = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int bb = 0; bb < 3; ++bb) pp += P[a][bb] * P[a][bb];
  const double Q = sqrt(2.0 * pp);
  const double c2 = (cs * delta) * (cs * delta);
  return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * c2 * Q / rho));
}

/* Conservation layer (SI section 2, "Neural Network Architecture"):
 * ohat_i = o_i + k1 + k2 c_ix + k3 c_iy + k4 c_iz, k1 = -sum o / 19,
 * k_{2,3,4} = -sum o c_a / 10. */
void o3_project(const double *o, double *ohat) {
  double s = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int i = 0; i < 19; ++i) {
    s += o[i];
    sx += o[i] * O3_CX[i];
    sy += o[i] * O3_CY[i];
    sz += o[i] * O3_CZ[i];
  }
  const double k1 = -s / 19.0, k2 = -sx / 10.0, k3 = -sy / 10.0, k4 = -sz / 10.0;
  for (int i = 0; i < 19; ++i)
    ohat[i] = o[i] + k1 + k2 * O3_CX[i] + k3 * O3_CY[i] + k4 * O3_CZ[i];
}

/* Packed weights: W1[h1][19], b1, W2[h2][h1], b2, W3[h3][h2], b3, W4[19][h3], b4. */
int o3_mlp_nparams(int h1, int h2, int h3) {
  return h1 * 19 + h1 + h2 * h1 + h2 + h3 * h2 + h3 + 19 * h3 + 19;
}

static double leaky(double a, double slope) { return a >= 0.0 ? a : slope * a; }

/* One dense layer: y_j = act(b_j + sum_k W[j][k] x_k). */
static void dense(const double *W, const double *bias, int nout, int nin, const double *x,
                  double *y, int act, double slope) {
  for (int j = 0; j < nout; ++j) {
    double a = bias[j];
    for (int k = 0; k < nin; ++k) a += W[(size_t)j * nin + k] * x[k];
    y[j] = act ? leaky(a, slope) : a;
  }
}

/* MLP 19 -> h1 -> h2 -> h3 -> 19, LeakyReLU on the hidden layers, linear output. */
void o3_mlp_forward(const double *theta, const o3_params *p, const double *x, double *o) {
  const int h1 = p->h1, h2 = p->h2, h3 = p->h3;
  const double *W1 = theta, *b1 = W1 + h1 * 19, *W2 = b1 + h1, *b2 = W2 + (size_t)h2 * h1;
  const double *W3 = b2 + h2, *b3 = W3 + (size_t)h3 * h2, *W4 = b3 + h3, *b4 = W4 + 19 * h3;
  double *a1 = (double *)malloc(sizeof(double) * (h1 + h2 + h3));
  double *a2 = a1 + h1, *a3 = a2 + h2;
  dense(W1, b1, h1, 19, x, a1, 1, p->leaky_slope);
  dense(W2, b2, h2, h1, a1, a2, 1, p->leaky_slope);
  dense(W3, b3, h3, h2, a2, a3, 1, p->leaky_slope);
  dense(W4, b4, 19, h3, a3, o, 0, 0.0);
  free(a1);
}

/* One node's collision, forcing applied last:
 *   BGK  f + (feq - f)/tau + f_ext                                  (Eq. S3, S5)
 *   SMAG f + (feq - f)/tau_eff + f_ext                              (SI sec. 1)
 *   MLP  f + (feq - f)/tau + (rho/tau) P[MLP((f - feq)/rho)] + f_ext (the learned model) */
void o3_collide_node(int kind, const double *f, double *post, const o3_params *p,
                     const double *theta, const double *F) {
  double rho, u[3], feq[19], fext[19];
  o3_node_moments(f, &rho, u);
  o3_feq(rho, u[0], u[1], u[2], feq);
  o3_edm_force(rho, u, F, fext);
  double tau = p->tau;
  if (kind == O3_SMAG) tau = o3_smag_tau_eff(f, p->tau, p->smag_cs, p->smag_delta);
  for (int i = 0; i < 19; ++i) post[i] = f[i] + (feq[i] - f[i]) / tau;
  if (kind == O3_MLP) {
    double x[19], o[19], oh[19];
    for (int i = 0; i < 19; ++i) x[i] = (f[i] - feq[i]) / rho;
    o3_mlp_forward(theta, p, x, o);
    o3_project(o, oh);
    for (int i = 0; i < 19; ++i) post[i] += (rho / p->tau) * oh[i];
  }
  for (int i = 0; i < 19; ++i) post[i] += fext[i];
}

void o3_collide(int B, int nz, int ny, int nx, int kind, const double *fpre, double *fpost,
                const o3_params *p, const double *theta) {
  for (int b = 0; b < B; ++b)
#pragma omp parallel for
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double f[19], q[19], F[3];
          o3_force(p, z, y, x, nz, ny, nx, F);
          for (int i = 0; i < 19; ++i) f[i] = fpre[idx5(b, i, z, y, x, nz, ny, nx)];
          o3_collide_node(kind, f, q, p, theta, F);
          for (int i = 0; i < 19; ++i) fpost[idx5(b, i, z, y, x, nz, ny, nx)] = q[i];
        }
}

/* g_out = C(S g_in): one step on the stored post-collision state. */
void o3_step(int B, int nz, int ny, int nx, int kind, const double *g_in, double *g_out,
             const o3_params *p, const double *theta) {
  const size_t n = (size_t)B * 19 * nz * ny * nx;
  double *f = (double *)malloc(sizeof(double) * n);
  o3_stream_pull(B, nz, ny, nx, g_in, f);
  o3_collide(B, nz, ny, nx, kind, f, g_out, p, theta);
  free(f);
}

void o3_run(int B, int nz, int ny, int nx, int kind, double *g, int nsteps, const o3_params *p,
            const double *theta) {
  const size_t n = (size_t)B * 19 * nz * ny * nx;
  double *t = (double *)malloc(sizeof(double) * n);
  for (int s = 0; s < nsteps; ++s) {
    o3_step(B, nz, ny, nx, kind, g, t, p, theta);
    memcpy(g, t, sizeof(double) * n);
  }
  free(t);
}

/* Equilibrium populations of given fields: rho [B][nz][ny][nx], u [B][3][nz][ny][nx]. */
void o3_feq_field(int B, int nz, int ny, int nx, const double *rho, const double *u,
                  double *f) {
  const size_t N = (size_t)nz * ny * nx;
  for (int b = 0; b < B; ++b)
    for (size_t n = 0; n < N; ++n) {
      double q[19];
      o3_feq(rho[(size_t)b * N + n], u[((size_t)b * 3 + 0) * N + n],
             u[((size_t)b * 3 + 1) * N + n], u[((size_t)b * 3 + 2) * N + n], q);
      for (int i = 0; i < 19; ++i) f[((size_t)b * 19 + i) * N + n] = q[i];
    }
}
