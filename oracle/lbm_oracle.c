/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the D2Q9 lattice-Boltzmann
 * hot path (stream, moments, equilibrium, BGK, Smagorinsky-BGK, learned
 * MLP collision with conservation projection, EDM forcing, box filter,
 * velocity loss and the hand-written reverse-mode adjoint of the unroll).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path calls this file;
 * it is loaded by the tests, by the smoke check and by the CPU-baseline leg
 * of the benchmark.  It shares no code, header or table with the CUDA path:
 * the lattice tables below are its own copy.
 *
 * Conventions
 *   - populations are SoA, index [b][i][y][x], x fastest;
 *   - every node loop is a plain loop over (b, y, x) (OpenMP over rows);
 *   - the stored state of a run is the POST-collision populations g at time
 *     t (pull scheme); the pre-collision populations at t+1 are the gathered
 *     values f_i(x) = g_i(x - c_i)  (stream/collide split, Methods, and the
 *     lattice Boltzmann equation, Eq. S2);
 *   - Delta t = Delta x = 1 throughout.
 *
 * Parity status of each function (what pins it is in tests/test_oracle_*.py):
 *   pinned: lattice, feq, stream, moments, bgk, smagorinsky, edm forcing,
 *           projection, mlp collision, box filter, loss, adjoint (FD).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 lattice: c_i and w_i (D2Q9 analogue of Tab. S1's D3Q19 stencil). */
static const int ORA_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ORA_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double ORA_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double ORA_CS2 = 1.0 / 3.0; /* c_s = 1/sqrt(3) */

enum { ORA_BGK = 0, ORA_SMAG = 1, ORA_MLP = 2 };

/* Collision parameters shared by every kind. */
typedef struct {
  double tau;        /* relaxation time (Eq. S3) */
  double smag_cs;    /* Smagorinsky constant C_s (Eq. S7) */
  double smag_delta; /* filter width Delta in lattice units */
  double force_amp;  /* Kolmogorov forcing amplitude F0 */
  int force_mode;    /* forcing wavenumber m: F_x(y) = F0 sin(2 pi m y / ny) */
  int hidden;        /* MLP hidden width (both hidden layers) */
} ora_params;

static inline size_t idx4(int b, int i, int y, int x, int ny, int nx) {
  return (((size_t)b * 9 + i) * ny + y) * nx + x;
}
static inline int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

void ora_lattice(int *cx, int *cy, double *w) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = ORA_CX[i];
    cy[i] = ORA_CY[i];
    w[i] = ORA_W[i];
  }
}

/* nu = c_s^2 (tau - dt/2), Eq. S6. */
double ora_viscosity(double tau) { return ORA_CS2 * (tau - 0.5); }

/* tau' = (tau - 1/2)/cg + 1/2, Eq. S9. */
double ora_tau_rescaled(double tau, double cg) { return (tau - 0.5) / cg + 0.5; }

/* Second-order equilibrium, Eq. S4:
 * feq_i = w_i rho (1 + u.c/cs^2 + ((u.c)^2 - cs^2 |u|^2) / (2 cs^4)). */
void ora_feq(double rho, double ux, double uy, double *feq) {
  const double usq = ux * ux + uy * uy;
  for (int i = 0; i < 9; ++i) {
    const double cu = ORA_CX[i] * ux + ORA_CY[i] * uy;
    feq[i] = ORA_W[i] * rho *
             (1.0 + cu / ORA_CS2 + (cu * cu - ORA_CS2 * usq) / (2.0 * ORA_CS2 * ORA_CS2));
  }
}

/* rho = sum f_i, rho u = sum f_i c_i  (SI section 1). */
static void node_moments(const double *f, double *rho, double *ux, double *uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    r += f[i];
    jx += f[i] * ORA_CX[i];
    jy += f[i] * ORA_CY[i];
  }
  *rho = r;
  *ux = jx / r;
  *uy = jy / r;
}

/* Streaming (pull): f_i(x) = g_i(x - c_i), stream/collide split (Methods). */
void ora_stream_pull(int B, int ny, int nx, const double *g, double *f) {
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 9; ++i)
#pragma omp parallel for
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          f[idx4(b, i, y, x, ny, nx)] =
              g[idx4(b, i, wrap(y - ORA_CY[i], ny), wrap(x - ORA_CX[i], nx), ny, nx)];
}

/* Anti-streaming (the inverse and transpose of the pull): g_i(x) = f_i(x + c_i),
 * i.e. streaming along -c_i (dataset construction step 4, SI section 2). */
void ora_stream_push(int B, int ny, int nx, const double *f, double *g) {
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 9; ++i)
#pragma omp parallel for
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          g[idx4(b, i, y, x, ny, nx)] =
              f[idx4(b, i, wrap(y + ORA_CY[i], ny), wrap(x + ORA_CX[i], nx), ny, nx)];
}

/* Per-node moments of a population field: rho, u = j / rho. */
void ora_moments(int B, int ny, int nx, const double *f, double *rho, double *ux,
                 double *uy) {
  for (int b = 0; b < B; ++b)
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double fn[9];
        for (int i = 0; i < 9; ++i) fn[i] = f[idx4(b, i, y, x, ny, nx)];
        const size_t n = ((size_t)b * ny + y) * nx + x;
        node_moments(fn, &rho[n], &ux[n], &uy[n]);
      }
}

/* Kolmogorov forcing used by every config: F = (F0 sin(2 pi m y / ny), 0). */
static double force_x(const ora_params *p, int y, int ny) {
  if (p->force_amp == 0.0) return 0.0;
  return p->force_amp * sin(2.0 * M_PI * (double)p->force_mode * (double)y / (double)ny);
}

/* Exact Difference Method forcing, Eq. S5:
 * f_ext_i = feq_i(rho, u + F/rho) - feq_i(rho, u). */
void ora_edm_force(double rho, double ux, double uy, double Fx, double Fy, double *fext) {
  double a[9], s[9];
  ora_feq(rho, ux, uy, a);
  ora_feq(rho, ux + Fx / rho, uy + Fy / rho, s);
  for (int i = 0; i < 9; ++i) fext[i] = s[i] - a[i];
}

/* Smagorinsky relaxation time (SI section 1, "Implementing the Smagorinsky
 * turbulence model in LBM").  Pi^neq_ab = sum_i c_ia c_ib (f_i - feq_i);
 * the strain follows from the Chapman-Enskog relation
 * S = -Pi^neq / (2 rho cs^2 tau_eff), |S| = sqrt(2 S:S);
 * nu_eff = nu0 + (C_s Delta)^2 |S| and tau_eff = nu_eff / cs^2 + 1/2 give the
 * quadratic tau_eff^2 - tau0 tau_eff - 9 (C_s Delta)^2 Q / (2 rho) = 0 with
 * Q = sqrt(2 Pi:Pi), whose positive root is returned. */
double ora_smag_tau_eff(const double *f, double tau0, double cs, double delta) {
  double rho, ux, uy, feq[9];
  node_moments(f, &rho, &ux, &uy);
  ora_feq(rho, ux, uy, feq);
  double pxx = 0.0, pxy = 0.0, pyy = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double d = f[i] - feq[i];
    pxx += ORA_CX[i] * ORA_CX[i] * d;
    pxy += ORA_CX[i] * ORA_CY[i] * d;
    pyy += ORA_CY[i] * ORA_CY[i] * d;
  }
  const double Q = sqrt(2.0 * (pxx * pxx + 2.0 * pxy * pxy + pyy * pyy));
  const double c2 = (cs * delta) * (cs * delta);
  return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * c2 * Q / rho));
}

/* Conservation projection, Eqs. S11-S12 written for D2Q9:
 * ohat_i = o_i + k1 + k2 c_ix + k3 c_iy with k1 = -sum o / 9 and
 * k_a = -sum o c_a / 6 (Q = 9 velocities, sum_i c_ia^2 = 6). */
void ora_project(const double *o, double *ohat) {
  double s = 0.0, sx = 0.0, sy = 0.0;
  for (int i = 0; i < 9; ++i) {
    s += o[i];
    sx += o[i] * ORA_CX[i];
    sy += o[i] * ORA_CY[i];
  }
  const double k1 = -s / 9.0, k2 = -sx / 6.0, k3 = -sy / 6.0;
  for (int i = 0; i < 9; ++i) ohat[i] = o[i] + k1 + k2 * ORA_CX[i] + k3 * ORA_CY[i];
}

/* Packed weight layout: W1[h][9], b1[h], W2[h][h], b2[h], W3[9][h], b3[9]. */
int ora_mlp_nparams(int h) { return h * 9 + h + h * h + h + 9 * h + 9; }

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  int h;
} mlp_view;

static mlp_view mlp_unpack(const double *theta, int h) {
  mlp_view m;
  m.h = h;
  m.W1 = theta;
  m.b1 = m.W1 + h * 9;
  m.W2 = m.b1 + h;
  m.b2 = m.W2 + h * h;
  m.W3 = m.b2 + h;
  m.b3 = m.W3 + 9 * h;
  return m;
}

/* MLP 9 -> h -> h -> 9, tanh hidden activations, linear output (SI section 2,
 * "Neural Network Architecture", with the widths and activation of this
 * build).  h1, h2 may be NULL; when given they receive the activations. */
static void mlp_forward(const mlp_view *m, const double *x, double *o, double *h1o,
                        double *h2o) {
  const int h = m->h;
  double h1[h], h2[h];
  for (int j = 0; j < h; ++j) {
    double a = m->b1[j];
    for (int k = 0; k < 9; ++k) a += m->W1[j * 9 + k] * x[k];
    h1[j] = tanh(a);
  }
  for (int j = 0; j < h; ++j) {
    double a = m->b2[j];
    for (int k = 0; k < h; ++k) a += m->W2[j * h + k] * h1[k];
    h2[j] = tanh(a);
  }
  for (int i = 0; i < 9; ++i) {
    double a = m->b3[i];
    for (int k = 0; k < h; ++k) a += m->W3[i * h + k] * h2[k];
    o[i] = a;
  }
  if (h1o) memcpy(h1o, h1, sizeof(double) * h);
  if (h2o) memcpy(h2o, h2, sizeof(double) * h);
}

void ora_mlp_forward(const double *theta, int h, const double *x, double *o) {
  mlp_view m = mlp_unpack(theta, h);
  mlp_forward(&m, x, o, NULL, NULL);
}

/* One node's collision (all kinds), forcing applied last:
 *   BGK         f_post = f + (feq - f)/tau + f_ext                 (Eq. S3, S5)
 *   Smagorinsky f_post = f + (feq - f)/tau_eff + f_ext             (SI sec. 1)
 *   MLP         f_post = f + (feq - f)/tau + (rho/tau) P[MLP(x)] + f_ext,
 *               x = (f - feq)/rho                                   (Eq. S10-S12)
 * Fx, Fy is the body force at this node. */
void ora_collide_node(int kind, const double *f, double *post, const ora_params *p,
                      const double *theta, double Fx, double Fy) {
  double rho, ux, uy, feq[9], fext[9];
  node_moments(f, &rho, &ux, &uy);
  ora_feq(rho, ux, uy, feq);
  ora_edm_force(rho, ux, uy, Fx, Fy, fext);
  double tau = p->tau;
  if (kind == ORA_SMAG) tau = ora_smag_tau_eff(f, p->tau, p->smag_cs, p->smag_delta);
  for (int i = 0; i < 9; ++i) post[i] = f[i] + (feq[i] - f[i]) / tau;
  if (kind == ORA_MLP) {
    double x[9], o[9], oh[9];
    for (int i = 0; i < 9; ++i) x[i] = (f[i] - feq[i]) / rho;
    mlp_view m = mlp_unpack(theta, p->hidden);
    mlp_forward(&m, x, o, NULL, NULL);
    ora_project(o, oh);
    for (int i = 0; i < 9; ++i) post[i] += (rho / p->tau) * oh[i];
  }
  for (int i = 0; i < 9; ++i) post[i] += fext[i];
}

/* Collide a whole pre-collision field. */
void ora_collide(int B, int ny, int nx, int kind, const double *fpre, double *fpost,
                 const ora_params *p, const double *theta) {
  for (int b = 0; b < B; ++b)
#pragma omp parallel for
    for (int y = 0; y < ny; ++y) {
      const double Fx = force_x(p, y, ny);
      for (int x = 0; x < nx; ++x) {
        double f[9], q[9];
        for (int i = 0; i < 9; ++i) f[i] = fpre[idx4(b, i, y, x, ny, nx)];
        ora_collide_node(kind, f, q, p, theta, Fx, 0.0);
        for (int i = 0; i < 9; ++i) fpost[idx4(b, i, y, x, ny, nx)] = q[i];
      }
    }
}

/* One lattice-Boltzmann step on the stored post-collision state:
 * g_out = C(S g_in)  (Eq. S2 with the stream/collide split). */
void ora_step(int B, int ny, int nx, int kind, const double *g_in, double *g_out,
              const ora_params *p, const double *theta) {
  const size_t n = (size_t)B * 9 * ny * nx;
  double *f = (double *)malloc(sizeof(double) * n);
  ora_stream_pull(B, ny, nx, g_in, f);
  ora_collide(B, ny, nx, kind, f, g_out, p, theta);
  free(f);
}

/* nsteps steps, in place on g. */
void ora_run(int B, int ny, int nx, int kind, double *g, int nsteps, const ora_params *p,
             const double *theta) {
  const size_t n = (size_t)B * 9 * ny * nx;
  double *t = (double *)malloc(sizeof(double) * n);
  for (int s = 0; s < nsteps; ++s) {
    ora_step(B, ny, nx, kind, g, t, p, theta);
    memcpy(g, t, sizeof(double) * n);
  }
  free(t);
}

/* Box filter of pre-collision fine populations onto the coarse grid: each
 * coarse node (I, J) takes, per i, the mean over the cg x cg fine block
 * {cg I .. cg I + cg - 1} x {cg J .. cg J + cg - 1}.  (Coarse-graining
 * filter phi of SI section 2, with a box average in place of subsampling.) */
void ora_box_filter(int B, int ny, int nx, int cg, const double *ffine, double *fcoarse) {
  const int NY = ny / cg, NX = nx / cg;
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 9; ++i)
#pragma omp parallel for
      for (int J = 0; J < NY; ++J)
        for (int I = 0; I < NX; ++I) {
          double s = 0.0;
          for (int a = 0; a < cg; ++a)
            for (int c = 0; c < cg; ++c) s += ffine[idx4(b, i, J * cg + a, I * cg + c, ny, nx)];
          fcoarse[idx4(b, i, J, I, NY, NX)] = s / (double)(cg * cg);
        }
}

/* Velocity loss L = 1/(2 N B) sum_{b,x} |u(x) - u_t(x)|^2 with u = j/rho of the
 * given pre-collision populations (the velocity form of Eq. S13 used here). */
double ora_velocity_loss(int B, int ny, int nx, const double *fpre, const double *utx,
                         const double *uty) {
  const size_t N = (size_t)ny * nx;
  double L = 0.0;
  for (int b = 0; b < B; ++b)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double f[9], rho, ux, uy;
        for (int i = 0; i < 9; ++i) f[i] = fpre[idx4(b, i, y, x, ny, nx)];
        node_moments(f, &rho, &ux, &uy);
        const size_t n = (size_t)b * N + (size_t)y * nx + x;
        const double dx = ux - utx[n], dy = uy - uty[n];
        L += dx * dx + dy * dy;
      }
  return L / (2.0 * (double)N * (double)B);
}

/* dL/df_i = (1/(N B)) [(u - u_t) . (c_i - u)] / rho. */
void ora_velocity_loss_grad(int B, int ny, int nx, const double *fpre, const double *utx,
                            const double *uty, double *dLdf) {
  const size_t N = (size_t)ny * nx;
  const double s = 1.0 / ((double)N * (double)B);
  for (int b = 0; b < B; ++b)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double f[9], rho, ux, uy;
        for (int i = 0; i < 9; ++i) f[i] = fpre[idx4(b, i, y, x, ny, nx)];
        node_moments(f, &rho, &ux, &uy);
        const size_t n = (size_t)b * N + (size_t)y * nx + x;
        const double dx = ux - utx[n], dy = uy - uty[n];
        for (int i = 0; i < 9; ++i)
          dLdf[idx4(b, i, y, x, ny, nx)] =
              s * (dx * (ORA_CX[i] - ux) + dy * (ORA_CY[i] - uy)) / rho;
      }
}

/* ---------------------------------------------------------------------------
 * Reverse mode of the learned collision at one node.  Given the node's
 * pre-collision populations f and the adjoint pb = dL/df_post, add
 * dL/df_pre to fb and the weight gradient to dtheta (same packed layout).
 * Each line is the transpose of one forward line of ora_collide_node.
 * ------------------------------------------------------------------------- */
static void feq_partials(double rho, double ux, double uy, int i, double *dr, double *dux,
                         double *duy) {
  /* feq_i = w_i rho (1 + 3 cu + 4.5 cu^2 - 1.5 |u|^2) */
  const double cu = ORA_CX[i] * ux + ORA_CY[i] * uy;
  const double usq = ux * ux + uy * uy;
  *dr = ORA_W[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  *dux = ORA_W[i] * rho * (3.0 * ORA_CX[i] + 9.0 * cu * ORA_CX[i] - 3.0 * ux);
  *duy = ORA_W[i] * rho * (3.0 * ORA_CY[i] + 9.0 * cu * ORA_CY[i] - 3.0 * uy);
}

static void mlp_collide_node_vjp(const double *f, const double *pb, const ora_params *p,
                                 const mlp_view *m, double Fx, double Fy, double *fb,
                                 double *dtheta) {
  const int h = m->h;
  const double tau = p->tau;
  double rho, ux, uy, feq[9], x[9], o[9], oh[9];
  node_moments(f, &rho, &ux, &uy);
  ora_feq(rho, ux, uy, feq);
  for (int i = 0; i < 9; ++i) x[i] = (f[i] - feq[i]) / rho;
  double h1[h], h2[h], a2b[h], a1b[h];
  mlp_forward(m, x, o, h1, h2);
  ora_project(o, oh);

  double rhob = 0.0, uxb = 0.0, uyb = 0.0;
  double feqb[9], ohb[9], ob[9], xb[9];
  /* post = f + (feq - f)/tau + (rho/tau) oh + fs - feq, fs = feq(rho, u + F/rho) */
  for (int i = 0; i < 9; ++i) {
    fb[i] += pb[i] * (1.0 - 1.0 / tau);
    feqb[i] = pb[i] / tau - pb[i];
    ohb[i] = (rho / tau) * pb[i];
    rhob += pb[i] * oh[i] / tau;
  }
  /* shifted equilibrium fs(rho, ux + Fx/rho, uy + Fy/rho) */
  {
    const double sx = ux + Fx / rho, sy = uy + Fy / rho;
    for (int i = 0; i < 9; ++i) {
      double dr, dux, duy;
      feq_partials(rho, sx, sy, i, &dr, &dux, &duy);
      rhob += pb[i] * (dr - dux * Fx / (rho * rho) - duy * Fy / (rho * rho));
      uxb += pb[i] * dux;
      uyb += pb[i] * duy;
    }
  }
  /* projection is symmetric: ob = P ohb */
  ora_project(ohb, ob);
  /* output layer */
  double *W3b = dtheta + (size_t)(m->W3 - m->W1);
  double *b3b = dtheta + (size_t)(m->b3 - m->W1);
  double *W2b = dtheta + (size_t)(m->W2 - m->W1);
  double *b2b = dtheta + (size_t)(m->b2 - m->W1);
  double *W1b = dtheta;
  double *b1b = dtheta + (size_t)(m->b1 - m->W1);
  for (int i = 0; i < 9; ++i) {
    b3b[i] += ob[i];
    for (int k = 0; k < h; ++k) W3b[i * h + k] += ob[i] * h2[k];
  }
  for (int k = 0; k < h; ++k) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += m->W3[i * h + k] * ob[i];
    a2b[k] = s * (1.0 - h2[k] * h2[k]);
  }
  for (int j = 0; j < h; ++j) {
    b2b[j] += a2b[j];
    for (int k = 0; k < h; ++k) W2b[j * h + k] += a2b[j] * h1[k];
  }
  for (int k = 0; k < h; ++k) {
    double s = 0.0;
    for (int j = 0; j < h; ++j) s += m->W2[j * h + k] * a2b[j];
    a1b[k] = s * (1.0 - h1[k] * h1[k]);
  }
  for (int j = 0; j < h; ++j) {
    b1b[j] += a1b[j];
    for (int k = 0; k < 9; ++k) W1b[j * 9 + k] += a1b[j] * x[k];
  }
  for (int k = 0; k < 9; ++k) {
    double s = 0.0;
    for (int j = 0; j < h; ++j) s += m->W1[j * 9 + k] * a1b[j];
    xb[k] = s;
  }
  /* x_i = (f_i - feq_i) / rho */
  for (int i = 0; i < 9; ++i) {
    fb[i] += xb[i] / rho;
    feqb[i] -= xb[i] / rho;
    rhob -= xb[i] * x[i] / rho;
  }
  /* feq(rho, u) */
  for (int i = 0; i < 9; ++i) {
    double dr, dux, duy;
    feq_partials(rho, ux, uy, i, &dr, &dux, &duy);
    rhob += feqb[i] * dr;
    uxb += feqb[i] * dux;
    uyb += feqb[i] * duy;
  }
  /* u = j / rho */
  const double jxb = uxb / rho, jyb = uyb / rho;
  rhob -= (uxb * ux + uyb * uy) / rho;
  /* rho = sum f, j = sum f c */
  for (int i = 0; i < 9; ++i) fb[i] += rhob + jxb * ORA_CX[i] + jyb * ORA_CY[i];
}

/* Loss of an unrolled learned-collision trajectory: start from the stored
 * post-collision state g0, take nsteps steps, stream once more to get the
 * pre-collision populations at the final time, and return the velocity
 * loss against (utx, uty)  (unrolled training, SI section 2). */
double ora_unroll_loss(int B, int ny, int nx, const double *g0, int nsteps,
                       const ora_params *p, const double *theta, const double *utx,
                       const double *uty) {
  const size_t n = (size_t)B * 9 * ny * nx;
  double *g = (double *)malloc(sizeof(double) * n);
  double *f = (double *)malloc(sizeof(double) * n);
  memcpy(g, g0, sizeof(double) * n);
  ora_run(B, ny, nx, ORA_MLP, g, nsteps, p, theta);
  ora_stream_pull(B, ny, nx, g, f);
  const double L = ora_velocity_loss(B, ny, nx, f, utx, uty);
  free(g);
  free(f);
  return L;
}

/* Hand-written reverse mode of ora_unroll_loss: returns L, writes
 * dL/dtheta (packed, overwritten) and, if dg0 != NULL, dL/dg0.
 * All intermediate states are kept (slow and simple). */
double ora_unroll_grad(int B, int ny, int nx, const double *g0, int nsteps,
                       const ora_params *p, const double *theta, const double *utx,
                       const double *uty, double *dtheta, double *dg0) {
  const size_t n = (size_t)B * 9 * ny * nx;
  const int np = ora_mlp_nparams(p->hidden);
  mlp_view m = mlp_unpack(theta, p->hidden);
  /* states g^0 .. g^nsteps */
  double *gs = (double *)malloc(sizeof(double) * n * (size_t)(nsteps + 1));
  memcpy(gs, g0, sizeof(double) * n);
  for (int s = 0; s < nsteps; ++s)
    ora_step(B, ny, nx, ORA_MLP, gs + n * s, gs + n * (s + 1), p, theta);
  double *f = (double *)malloc(sizeof(double) * n);
  double *lam_pre = (double *)malloc(sizeof(double) * n);
  double *lam = (double *)malloc(sizeof(double) * n);
  ora_stream_pull(B, ny, nx, gs + n * nsteps, f);
  const double L = ora_velocity_loss(B, ny, nx, f, utx, uty);
  ora_velocity_loss_grad(B, ny, nx, f, utx, uty, lam_pre);
  /* the transpose of the pull is the push */
  ora_stream_push(B, ny, nx, lam_pre, lam);
  memset(dtheta, 0, sizeof(double) * np);
  for (int s = nsteps - 1; s >= 0; --s) {
    /* g^{s+1} = C(S g^s): lam currently holds dL/dg^{s+1} */
    ora_stream_pull(B, ny, nx, gs + n * s, f);
    memset(lam_pre, 0, sizeof(double) * n);
    for (int b = 0; b < B; ++b)
      for (int y = 0; y < ny; ++y) {
        const double Fx = force_x(p, y, ny);
        for (int x = 0; x < nx; ++x) {
          double fn[9], pb[9], fb[9] = {0};
          for (int i = 0; i < 9; ++i) {
            fn[i] = f[idx4(b, i, y, x, ny, nx)];
            pb[i] = lam[idx4(b, i, y, x, ny, nx)];
          }
          mlp_collide_node_vjp(fn, pb, p, &m, Fx, 0.0, fb, dtheta);
          for (int i = 0; i < 9; ++i) lam_pre[idx4(b, i, y, x, ny, nx)] = fb[i];
        }
      }
    ora_stream_push(B, ny, nx, lam_pre, lam);
  }
  if (dg0) memcpy(dg0, lam, sizeof(double) * n);
  free(gs);
  free(f);
  free(lam_pre);
  free(lam);
  return L;
}

/* Single-node vjp exposed for tests. */
void ora_mlp_collide_vjp(const double *f, const double *pb, const ora_params *p,
                         const double *theta, double Fx, double Fy, double *fb,
                         double *dtheta) {
  mlp_view m = mlp_unpack(theta, p->hidden);
  for (int i = 0; i < 9; ++i) fb[i] = 0.0;
  mlp_collide_node_vjp(f, pb, p, &m, Fx, Fy, fb, dtheta);
}

/* f = feq(rho, u) at every node of a (B, ny, nx) field (Eq. S4). */
void ora_feq_field(int B, int ny, int nx, const double *rho, const double *ux,
                   const double *uy, double *f) {
  for (int b = 0; b < B; ++b)
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t n = ((size_t)b * ny + y) * nx + x;
        double q[9];
        ora_feq(rho[n], ux[n], uy[n], q);
        for (int i = 0; i < 9; ++i) f[idx4(b, i, y, x, ny, nx)] = q[i];
      }
}

/* Longitudinal velocity structure functions (the paper's structure-function
 * definition, SI section 3): S^p(r) = < [(u(x + r e) - u(x)) . e]^p > for
 * p = 1..6 and r = 1..rmax, averaged over every node and over the two lattice
 * directions e = x^, y^ (periodic).  S is [6][rmax], S[(p-1)*rmax + r-1]. */
void ora_structure_functions(int B, int ny, int nx, const double *ux, const double *uy,
                             int rmax, double *S) {
  for (int k = 0; k < 6 * rmax; ++k) S[k] = 0.0;
  for (int r = 1; r <= rmax; ++r) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < B; ++b)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const size_t n = ((size_t)b * ny + y) * nx + x;
          const double dx = ux[((size_t)b * ny + y) * nx + (x + r) % nx] - ux[n];
          const double dy = uy[((size_t)b * ny + (y + r) % ny) * nx + x] - uy[n];
          double px = 1.0, py = 1.0;
          for (int p = 0; p < 6; ++p) {
            px *= dx;
            py *= dy;
            acc[p] += px + py;
          }
        }
    for (int p = 0; p < 6; ++p) S[p * rmax + r - 1] = acc[p] / (2.0 * B * ny * nx);
  }
}

/* Velocity loss on a subset of nodes (Eq. S13 with the random subset S of the
 * unrolled training, velocity form): idx are flat node indices b*ny*nx + y*nx + x;
 * L = 1/(2 |S|) sum_{n in S} |u(n) - u_t(n)|^2, u = j/rho of the given
 * pre-collision populations; dLdf (nullable, full field) gets the gradient. */
double ora_velocity_loss_subset(int B, int ny, int nx, const double *fpre, const int *idx,
                                int count, const double *utx, const double *uty, double *dLdf) {
  const size_t N = (size_t)ny * nx;
  if (dLdf)
    for (size_t k = 0; k < (size_t)B * 9 * N; ++k) dLdf[k] = 0.0;
  double L = 0.0;
  for (int s = 0; s < count; ++s) {
    const size_t n = (size_t)idx[s];
    const int b = (int)(n / N), y = (int)((n % N) / nx), x = (int)(n % nx);
    double f[9], rho, ux, uy;
    for (int i = 0; i < 9; ++i) f[i] = fpre[idx4(b, i, y, x, ny, nx)];
    node_moments(f, &rho, &ux, &uy);
    const double dx = ux - utx[n], dy = uy - uty[n];
    L += dx * dx + dy * dy;
    if (dLdf)
      for (int i = 0; i < 9; ++i)
        dLdf[idx4(b, i, y, x, ny, nx)] +=
            (dx * (ORA_CX[i] - ux) + dy * (ORA_CY[i] - uy)) / (rho * count);
  }
  return L / (2.0 * count);
}

/* Population loss of Eq. S13 on a subset S of nodes, as the paper writes it (a
 * plain sum, no normalisation): L = sum_{n in S} sum_i (g_i(n) - t_i(n))^2 for
 * post-collision populations g (the stored state) and targets t; dLdg
 * (nullable, full field) gets the gradient 2 (g - t) on S and 0 elsewhere.
 * A node listed twice counts twice. */
double ora_population_loss_subset(int B, int ny, int nx, const double *g, const int *idx,
                                  int count, const double *t, double *dLdg) {
  const size_t N = (size_t)ny * nx;
  if (dLdg)
    for (size_t k = 0; k < (size_t)B * 9 * N; ++k) dLdg[k] = 0.0;
  double L = 0.0;
  for (int s = 0; s < count; ++s) {
    const size_t n = (size_t)idx[s];
    const int b = (int)(n / N), y = (int)((n % N) / nx), x = (int)(n % nx);
    for (int i = 0; i < 9; ++i) {
      const size_t k = idx4(b, i, y, x, ny, nx);
      const double d = g[k] - t[k];
      L += d * d;
      if (dLdg) dLdg[k] += 2.0 * d;
    }
  }
  return L;
}

/* Coarse-graining by subsampling (SI section 2, filter phi): f_c(I, J) = f(cg I, cg J). */
void ora_subsample(int B, int ny, int nx, int cg, const double *f, double *fc) {
  const int NY = ny / cg, NX = nx / cg;
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < 9; ++i)
      for (int J = 0; J < NY; ++J)
        for (int I = 0; I < NX; ++I)
          fc[idx4(b, i, J, I, NY, NX)] = f[idx4(b, i, J * cg, I * cg, ny, nx)];
}
