/*
 * gpmood_oracle.c -- plain, slow FP64 CPU oracle of GP-MOOD (arXiv:2110.08683).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  Independent of the
 * CUDA implementation: nothing here is shared with it.
 *
 * The code follows the paper's definitions in the paper's order:
 *   Sec. 2.1  Euler equations, EoS, FV update (eq. fvm_discrete, eq. fvm_F)
 *   Sec. 2.2  GP stencil (blocky diamond), Table QR (Gauss rules)
 *   Sec. 2.4  volume-averaged SE kernels (eq. SE-pred, SE-cov, delta_mnd),
 *             prediction vector (eq. gp_reconstructor) and its normalisation
 *             (eq. normalized_z), Cholesky solve
 *   Sec. 2.5  weights in quadruple precision, stored in double
 *   Sec. 2.6  FOG = radius 0
 *   Sec. 3.1 (iv), App. C  Poly3 of POL-MOOD3 (eq. poly3, eq. p3_coeffs)
 *   Sec. 3.2-3.4  PAD, CAD (cell and face states), plateau, DMP, u2, CSD
 *   Sec. 3.6  EDP1 face orders
 *   Sec. 3.8  SSP-RK3 (eq. rk3)
 *   Sec. 4    Steps 1-10
 *   App. B    GP second-derivative weights
 * Where the paper leaves a point open, the reading taken is stated in a
 * comment at the code it shapes (for example: z normalised by its signed sum
 * so that z^T 1 = 1; the diamond |a|+|b| <= R stencil; the per-direction CFL
 * bound; density alone in DMP, plateau and u2; the queued cells and their
 * face neighbours re-detected after each MOOD iteration).
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "gpmood_oracle.h"

typedef _Float128 qreal;

#define NV 4          /* conservative variables */
#define MAXN 25       /* largest stencil: R = 3 diamond */
#define MAXQ 4

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rules on the reference face [-1/2, 1/2]  (Table QR)          */
/* ------------------------------------------------------------------------- */
static void gauss_rule_q(int q, qreal* g, qreal* w) {
  if (q == 1) {
    g[0] = 0; w[0] = 1;
  } else if (q == 2) {
    qreal a = 1 / (2 * sqrtf128(3));
    g[0] = a; g[1] = -a;
    w[0] = w[1] = (qreal)1 / 2;
  } else if (q == 3) {
    qreal a = sqrtf128((qreal)3 / 5) / 2;
    g[0] = a; g[1] = 0; g[2] = -a;
    w[0] = (qreal)5 / 18; w[1] = (qreal)8 / 18; w[2] = (qreal)5 / 18;
  } else {
    qreal r = 2 * sqrtf128((qreal)6 / 5) / 7;
    qreal a = sqrtf128((qreal)3 / 7 + r) / 2;
    qreal b = sqrtf128((qreal)3 / 7 - r) / 2;
    g[0] = a; g[1] = b; g[2] = -b; g[3] = -a;
    qreal s30 = sqrtf128(30);
    w[0] = (18 - s30) / 72; w[1] = (18 + s30) / 72;
    w[2] = (18 + s30) / 72; w[3] = (18 - s30) / 72;
  }
}

int orc_gauss_rule(int q, double* g, double* w) {
  if (q < 1 || q > 4) return -1;
  qreal gq[MAXQ], wq[MAXQ];
  gauss_rule_q(q, gq, wq);
  for (int k = 0; k < q; ++k) { g[k] = (double)gq[k]; w[k] = (double)wq[k]; }
  return q;
}

/* number of Gauss points used by a face reconstructed at radius R
   (Sec. 4 Step 3: R1 -> 2, R2 -> 3, R3 -> 4; FOG -> 1) */
static int face_q(int dim, int R) {
  if (dim == 1 || R == 0) return 1;
  return R + 1;
}

/* ------------------------------------------------------------------------- */
/* GP stencil of radius R: the cells with |a| + |b| <= R (Sec. 2.2).           */
/* Centre first, then ring by ring; ring r starts at (-r,0) and runs through   */
/* (0,r), (r,0), (0,-r).  For R = 1 this is the labelling of App. A:           */
/* 1 = centre, 2 = west, 3 = north, 4 = east, 5 = south.                      */
/* ------------------------------------------------------------------------- */
int orc_stencil(int dim, int R, int* off) {
  int n = 0;
  off[0] = 0; off[1] = 0; n = 1;
  for (int r = 1; r <= R; ++r) {
    if (dim == 1) {
      off[2 * n] = -r; off[2 * n + 1] = 0; ++n;
      off[2 * n] = r; off[2 * n + 1] = 0; ++n;
      continue;
    }
    for (int k = 0; k < r; ++k) { off[2 * n] = -r + k; off[2 * n + 1] = k; ++n; }
    for (int k = 0; k < r; ++k) { off[2 * n] = k; off[2 * n + 1] = r - k; ++n; }
    for (int k = 0; k < r; ++k) { off[2 * n] = r - k; off[2 * n + 1] = -k; ++n; }
    for (int k = 0; k < r; ++k) { off[2 * n] = -k; off[2 * n + 1] = -r + k; ++n; }
  }
  return n;
}

/* ------------------------------------------------------------------------- */
/* Volume-averaged SE kernels in one dimension, in units of the cell size:     */
/* lam = ell / Delta_d and delta = Delta_{m*,d} or Delta_{mn,d} (eq. delta_mnd) */
/* ------------------------------------------------------------------------- */
static qreal q_pi(void) { return 4 * atanf128(1); }

/* one factor of eq. SE-pred */
static qreal pred_1d_q(qreal delta, qreal lam) {
  qreal s = sqrtf128(2) * lam;
  return sqrtf128(q_pi() / 2) * lam *
         (erff128((delta + (qreal)1 / 2) / s) - erff128((delta - (qreal)1 / 2) / s));
}

/* one factor of eq. SE-cov (the second erf argument divides by lam, as the
   first one does; the printed subscript d is missing there) */
static qreal cov_1d_q(qreal delta, qreal lam) {
  qreal s = sqrtf128(2) * lam;
  qreal sp = sqrtf128(q_pi());
  qreal up = (delta + 1) / s, um = (delta - 1) / s, u0 = delta / s;
  qreal t1 = up * erff128(up) + um * erff128(um);
  qreal t2 = (expf128(-(delta + 1) * (delta + 1) / (2 * lam * lam)) +
              expf128(-(delta - 1) * (delta - 1) / (2 * lam * lam))) / sp;
  qreal t3 = 2 * (u0 * erff128(u0) + expf128(-delta * delta / (2 * lam * lam)) / sp);
  return sp * lam * lam * (t1 + t2 - t3);
}

/* second derivative of one eq. SE-pred factor with respect to the physical
   coordinate of x_* (App. B); ell is physical, lam = ell / Delta_d */
static qreal pred_1d_d2_q(qreal delta, qreal lam, qreal ell) {
  qreal a = delta - (qreal)1 / 2, b = delta + (qreal)1 / 2;
  return (a * expf128(-a * a / (2 * lam * lam)) - b * expf128(-b * b / (2 * lam * lam))) /
         (ell * ell);
}

double orc_pred_1d(double delta, double lam) { return (double)pred_1d_q(delta, lam); }
double orc_cov_1d(double delta, double lam) { return (double)cov_1d_q(delta, lam); }

/* ------------------------------------------------------------------------- */
/* Cholesky solve of the SPD system C z = t in quad precision (Sec. 2.4-2.5)  */
/* ------------------------------------------------------------------------- */
static int cholesky_q(int n, qreal* C /* n*n, overwritten by L */) {
  for (int j = 0; j < n; ++j) {
    qreal d = C[j * n + j];
    for (int k = 0; k < j; ++k) d -= C[j * n + k] * C[j * n + k];
    if (!(d > 0)) return -1;
    qreal ljj = sqrtf128(d);
    C[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      qreal s = C[i * n + j];
      for (int k = 0; k < j; ++k) s -= C[i * n + k] * C[j * n + k];
      C[i * n + j] = s / ljj;
    }
  }
  return 0;
}

static void cholesky_solve_q(int n, const qreal* L, const qreal* t, qreal* z) {
  qreal y[MAXN];
  for (int i = 0; i < n; ++i) {
    qreal s = t[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    qreal s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * z[k];
    z[i] = s / L[i * n + i];
  }
}

/* covariance matrix C_mn of eq. SE-cov on the radius-R stencil */
static void build_cov_q(int dim, int n, const int* off, qreal lamx, qreal lamy, qreal* C) {
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k) {
      qreal dxm = (qreal)(off[2 * k] - off[2 * m]);
      qreal dym = (qreal)(off[2 * k + 1] - off[2 * m + 1]);
      qreal c = cov_1d_q(dxm, lamx);
      if (dim == 2) c *= cov_1d_q(dym, lamy);
      C[m * n + k] = c;
    }
}

/* face geometry: position of the Gauss point relative to the cell centre, in
   cell units.  face 0 = east (x=+1/2), 1 = west, 2 = north (y=+1/2), 3 = south;
   g runs along the face (y for E/W faces, x for N/S faces). */
static void face_point(int face, qreal g, qreal* xs, qreal* ys) {
  switch (face) {
  case 0: *xs = (qreal)1 / 2; *ys = g; break;
  case 1: *xs = -(qreal)1 / 2; *ys = g; break;
  case 2: *xs = g; *ys = (qreal)1 / 2; break;
  default: *xs = g; *ys = -(qreal)1 / 2; break;
  }
}

static int weights_impl(int dim, int R, double lamx_d, double lamy_d, double* zout,
                        int normalise, int* nq_out, int* nn_out) {
  if (R < 1 || R > 3 || (dim != 1 && dim != 2)) return -1;
  int off[2 * MAXN];
  int n = orc_stencil(dim, R, off);
  int q = face_q(dim, R);
  int nfaces = (dim == 2) ? 4 : 2;
  qreal lamx = lamx_d, lamy = lamy_d;
  qreal C[MAXN * MAXN], t[MAXN], z[MAXN];
  build_cov_q(dim, n, off, lamx, lamy, C);
  if (cholesky_q(n, C) != 0) return -2;
  qreal g[MAXQ], w[MAXQ];
  gauss_rule_q(q, g, w);
  for (int f = 0; f < nfaces; ++f)
    for (int gi = 0; gi < q; ++gi) {
      qreal xs, ys;
      face_point(f, (dim == 2) ? g[gi] : 0, &xs, &ys);
      for (int m = 0; m < n; ++m) {
        /* Delta_{m*,d} = e_d . (x_* - x_m) / Delta_d */
        qreal tm = pred_1d_q(xs - off[2 * m], lamx);
        if (dim == 2) tm *= pred_1d_q(ys - off[2 * m + 1], lamy);
        t[m] = tm;
      }
      cholesky_solve_q(n, C, t, z); /* z = C^{-1} t*, i.e. z^T = t*^T C^{-1} */
      qreal s = 0;
      for (int m = 0; m < n; ++m) s += z[m];
      for (int m = 0; m < n; ++m) {
        /* eq. normalized_z: divide by the (signed) sum so that z^T 1 = 1 */
        qreal zm = normalise ? z[m] / s : z[m];
        zout[(f * q + gi) * n + m] = (double)zm;
      }
    }
  if (nq_out) *nq_out = q;
  if (nn_out) *nn_out = n;
  return 0;
}

int orc_gp_weights(int dim, int R, double lamx, double lamy, double* z, int* nq, int* nn) {
  return weights_impl(dim, R, lamx, lamy, z, 1, nq, nn);
}

int orc_gp_weights_raw(int dim, int R, double lamx, double lamy, double* z) {
  return weights_impl(dim, R, lamx, lamy, z, 0, 0, 0);
}

/* App. B: d^2 t*_m / dx*^2 at the cell centre, then w = C^{-1} t'' (R = 1 stencil) */
int orc_d2_weights(int dim, double ell_d, double dx, double dy, double* wxx, double* wyy) {
  int off[2 * MAXN];
  int n = orc_stencil(dim, 1, off);
  qreal ell = ell_d, lamx = ell / (qreal)dx, lamy = ell / (qreal)dy;
  qreal C[MAXN * MAXN], t[MAXN] = {0}, z[MAXN];
  build_cov_q(dim, n, off, lamx, lamy, C);
  if (cholesky_q(n, C) != 0) return -2;
  for (int d = 0; d < dim; ++d) {
    for (int m = 0; m < n; ++m) {
      qreal dxm = -(qreal)off[2 * m], dym = -(qreal)off[2 * m + 1];
      qreal tm;
      if (d == 0) {
        tm = pred_1d_d2_q(dxm, lamx, ell);
        if (dim == 2) tm *= pred_1d_q(dym, lamy);
      } else {
        tm = pred_1d_q(dxm, lamx) * pred_1d_d2_q(dym, lamy, ell);
      }
      t[m] = tm;
    }
    cholesky_solve_q(n, C, t, z);
    for (int m = 0; m < n; ++m) (d == 0 ? wxx : wyy)[m] = (double)z[m];
  }
  if (dim == 1)
    for (int m = 0; m < n; ++m) wyy[m] = 0.0;
  return n;
}

/* ------------------------------------------------------------------------- */
/* Poly3 of POL-MOOD3 (Sec. 3.1 (iv)): p3 = a0 + a1 x + a2 x^2 + a3 y + a4 y^2  */
/* (+ a5 xy, eq. poly3) matched to the five cell averages of the R = 1 stencil  */
/* (eq. p3_coeffs).  The xy monomial averages to zero on each of the five     */
/* cells, so a5 is left at 0.  The coefficients are App. C's, with its        */
/* labelling q1 centre, q2 west, q3 north, q4 east, q5 south (the orc_stencil */
/* order), in cell units with the origin at the cell centre.                 */
/* ------------------------------------------------------------------------- */
static void poly3_coeffs(const double* q /* q1..q5 as q[0..4] */, double* a) {
  a[0] = 7.0 / 6.0 * q[0] - q[1] / 24.0 - q[2] / 24.0 - q[3] / 24.0 - q[4] / 24.0;
  a[1] = -0.5 * q[1] + 0.5 * q[3];
  a[2] = -q[0] + 0.5 * q[1] + 0.5 * q[3];
  a[3] = 0.5 * q[2] - 0.5 * q[4];
  a[4] = -q[0] + 0.5 * q[2] + 0.5 * q[4];
}

double orc_poly3_eval(int dim, const double* qv, double xs, double ys) {
  double q[5], a[5];
  if (dim == 1) {
    /* 1D stencil order: centre, west, east; the y neighbours equal the centre */
    q[0] = qv[0]; q[1] = qv[1]; q[2] = qv[0]; q[3] = qv[2]; q[4] = qv[0];
  } else {
    for (int m = 0; m < 5; ++m) q[m] = qv[m];
  }
  poly3_coeffs(q, a);
  return a[0] + a[1] * xs + a[2] * xs * xs + a[3] * ys + a[4] * ys * ys;
}

/* ------------------------------------------------------------------------- */
/* context                                                                   */
/* ------------------------------------------------------------------------- */
struct orc_ctx {
  orc_config cfg;
  int H, gx, gy;          /* ghost width and ghosted extents */
  double dx, dy;
  int top;                /* highest radius of the cascade */
  int n[4], q[4];
  int off[4][2 * MAXN];
  double* z[4];           /* z[R][face][g][m] */
  double gq[5][MAXQ], gw[5][MAXQ];
  int off1[2 * MAXN];
  double wxx[MAXN], wyy[MAXN];
  /* work buffers */
  double *Xg, *Fx, *Fy, *Y, *U0, *S;
  double *Us[5], *Fn, *F3;  /* SSP-RK4: U^(1..4), F_nabla of a stage, F_nabla(U^(3)) */
  uint8_t *ord, *cad, *bad, *first, *inA;
};

static size_t gidx(const orc_ctx* c, int v, int i, int j) {
  return ((size_t)v * c->gy + (size_t)(j + c->H)) * c->gx + (size_t)(i + c->H);
}
static size_t iidx(const orc_ctx* c, int v, int i, int j) {
  return ((size_t)v * c->cfg.ny + (size_t)j) * c->cfg.nx + (size_t)i;
}

int orc_ghost_width(const orc_ctx* ctx) { return ctx->H; }

int orc_create(const orc_config* cfg, orc_ctx** out) {
  *out = 0;
  if (cfg->dim != 1 && cfg->dim != 2) return -1;
  if (cfg->nx < 1 || cfg->ny < 1 || (cfg->dim == 1 && cfg->ny != 1)) return -1;
  if (cfg->ncascade < 1 || cfg->ncascade > 4) return -1;
  if (cfg->rk != 0 && cfg->rk != 3 && cfg->rk != 4) return -1;
  if (cfg->riemann != 0 && cfg->riemann != 1) return -1;
  if (cfg->cascade[cfg->ncascade - 1] != 0) return -1;
  for (int k = 0; k + 1 < cfg->ncascade; ++k)
    if (!(cfg->cascade[k] > cfg->cascade[k + 1])) return -1;
  if (cfg->cascade[0] > 3) return -1;
  if (cfg->poly3 && !(cfg->ncascade == 2 && cfg->cascade[0] == 1)) return -1;
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->cfg = *cfg;
  c->top = cfg->cascade[0];
  c->H = c->top + 1 > 2 ? c->top + 1 : 2;
  for (int s = 0; s < 4; ++s) {
    int k = cfg->bc[s];
    if (k < 0 || k > 6) { free(c); return -1; }
    if (k == ORC_BC_JET && s < 2) { free(c); return -1; }
    if (k == ORC_BC_DMR_BOTTOM && s != 2) { free(c); return -1; }
    if (k == ORC_BC_DMR_TOP && s != 3) { free(c); return -1; }
    if ((cfg->bc[0] == ORC_BC_PERIODIC) != (cfg->bc[1] == ORC_BC_PERIODIC)) { free(c); return -1; }
    if (cfg->dim == 2 && (cfg->bc[2] == ORC_BC_PERIODIC) != (cfg->bc[3] == ORC_BC_PERIODIC)) {
      free(c); return -1;
    }
  }
  /* mirrored ghosts need as many interior cells as ghost layers */
  if (cfg->nx < c->H && cfg->bc[0] != ORC_BC_PERIODIC) { free(c); return -1; }
  if (cfg->dim == 2 && cfg->ny < c->H && cfg->bc[2] != ORC_BC_PERIODIC) { free(c); return -1; }
  c->gx = cfg->nx + 2 * c->H;
  c->gy = cfg->ny + 2 * c->H;
  c->dx = (cfg->x1 - cfg->x0) / cfg->nx;
  c->dy = (cfg->dim == 2) ? (cfg->y1 - cfg->y0) / cfg->ny : c->dx;
  double lamx = cfg->ell / c->dx, lamy = cfg->ell / c->dy;
  for (int k = 0; k < cfg->ncascade; ++k) {
    int R = cfg->cascade[k];
    if (R == 0) continue;
    c->n[R] = orc_stencil(cfg->dim, R, c->off[R]);
    c->q[R] = face_q(cfg->dim, R);
    c->z[R] = (double*)malloc(sizeof(double) * 4 * MAXQ * MAXN);
    if (cfg->poly3) continue; /* Poly3 is evaluated from App. C, no weights */
    if (orc_gp_weights(cfg->dim, R, lamx, lamy, c->z[R], 0, 0) != 0) {
      orc_destroy(c);
      return -2;
    }
  }
  for (int q = 1; q <= 4; ++q) orc_gauss_rule(q, c->gq[q], c->gw[q]);
  orc_stencil(cfg->dim, 1, c->off1);
  if (cfg->poly3) {
    /* POL-MOOD3: the u2 curvatures (eq. u2_curvature) are p3's own second
       derivatives, 2 a2 / dx^2 and 2 a4 / dy^2 (App. C), i.e. the centred
       differences q2 - 2 q1 + q4 and q3 - 2 q1 + q5 over the cell size squared */
    int n1 = orc_stencil(cfg->dim, 1, c->off1);
    for (int m = 0; m < n1; ++m) {
      int a = c->off1[2 * m], b = c->off1[2 * m + 1];
      c->wxx[m] = (b == 0 ? (a == 0 ? -2.0 : 1.0) : 0.0) / (c->dx * c->dx);
      c->wyy[m] = (cfg->dim == 2 && a == 0) ? (b == 0 ? -2.0 : 1.0) / (c->dy * c->dy) : 0.0;
    }
  } else if (orc_d2_weights(cfg->dim, cfg->ell, c->dx, c->dy, c->wxx, c->wyy) < 0) {
    orc_destroy(c);
    return -2;
  }
  size_t ng = (size_t)NV * c->gx * c->gy, ni = (size_t)NV * cfg->nx * cfg->ny;
  size_t nc = (size_t)cfg->nx * cfg->ny;
  c->Xg = (double*)calloc(ng, sizeof(double));
  c->Fx = (double*)calloc((size_t)NV * cfg->ny * (cfg->nx + 1), sizeof(double));
  c->Fy = (double*)calloc((size_t)NV * (cfg->ny + 1) * cfg->nx, sizeof(double));
  c->Y = (double*)calloc(ni, sizeof(double));
  c->U0 = (double*)calloc(ni, sizeof(double));
  c->S = (double*)calloc(ni, sizeof(double));
  for (int s = 1; s < 5; ++s) c->Us[s] = (double*)calloc(ni, sizeof(double));
  c->Fn = (double*)calloc(ni, sizeof(double));
  c->F3 = (double*)calloc(ni, sizeof(double));
  c->ord = (uint8_t*)calloc(nc, 1);
  c->cad = (uint8_t*)calloc(nc, 1);
  c->bad = (uint8_t*)calloc(nc, 1);
  c->first = (uint8_t*)calloc(nc, 1);
  c->inA = (uint8_t*)calloc(nc, 1);
  *out = c;
  return 0;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  for (int R = 0; R < 4; ++R) free(c->z[R]);
  free(c->Xg); free(c->Fx); free(c->Fy); free(c->Y); free(c->U0); free(c->S);
  for (int s = 1; s < 5; ++s) free(c->Us[s]);
  free(c->Fn); free(c->F3);
  free(c->ord); free(c->cad); free(c->bad); free(c->first); free(c->inA);
  free(c);
}

/* ------------------------------------------------------------------------- */
/* Euler equations and ideal-gas EoS (Sec. 2.1)                               */
/* ------------------------------------------------------------------------- */
static double pressure(const double* U, double gam) {
  return (gam - 1.0) * (U[3] - 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

static void prim_to_cons(const double* P, double gam, double* U) {
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[0] * P[2];
  U[3] = P[3] / (gam - 1.0) + 0.5 * P[0] * (P[1] * P[1] + P[2] * P[2]);
}

static void hllc_y(const double* UL, const double* UR, double gam, double* G);
static double dmin2(double a, double b) { return a < b ? a : b; }
static double dmax2(double a, double b) { return a > b ? a : b; }

/* HLLC approximate Riemann solver in the x direction (Toro et al. 1994;
   wave speeds S_L = min(u_L-c_L, u_R-c_R), S_R = max(u_L+c_L, u_R+c_R)) */
static void hllc_x(const double* UL, const double* UR, double gam, double* F) {
  double rL = UL[0], uL = UL[1] / rL, vL = UL[2] / rL, EL = UL[3];
  double rR = UR[0], uR = UR[1] / rR, vR = UR[2] / rR, ER = UR[3];
  double pL = pressure(UL, gam), pR = pressure(UR, gam);
  double cL = sqrt(gam * pL / rL), cR = sqrt(gam * pR / rR);
  double SL = dmin2(uL - cL, uR - cR);
  double SR = dmax2(uL + cL, uR + cR);
  double num = pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR);
  double den = rL * (SL - uL) - rR * (SR - uR);
  double Ss = num / den;
  double FL[4] = {rL * uL, rL * uL * uL + pL, rL * uL * vL, uL * (EL + pL)};
  double FR[4] = {rR * uR, rR * uR * uR + pR, rR * uR * vR, uR * (ER + pR)};
  if (!(rL > 0.0 && rR > 0.0 && pL > 0.0 && pR > 0.0)) {
    /* a state outside the solver's domain (c^2 = gamma p / rho <= 0 or NaN):
       the flux is undefined */
    for (int v = 0; v < 4; ++v) F[v] = NAN;
  } else if (SL >= 0.0) {
    for (int v = 0; v < 4; ++v) F[v] = FL[v];
  } else if (Ss >= 0.0) {
    double f = rL * (SL - uL) / (SL - Ss);
    double Us[4] = {f, f * Ss, f * vL, f * (EL / rL + (Ss - uL) * (Ss + pL / (rL * (SL - uL))))};
    for (int v = 0; v < 4; ++v) F[v] = FL[v] + SL * (Us[v] - UL[v]);
  } else if (SR > 0.0) {
    double f = rR * (SR - uR) / (SR - Ss);
    double Us[4] = {f, f * Ss, f * vR, f * (ER / rR + (Ss - uR) * (Ss + pR / (rR * (SR - uR))))};
    for (int v = 0; v < 4; ++v) F[v] = FR[v] + SR * (Us[v] - UR[v]);
  } else {
    for (int v = 0; v < 4; ++v) F[v] = FR[v];
  }
}

void orc_hllc(const double* UL, const double* UR, double gam, int dir, double* F) {
  if (dir == 0) hllc_x(UL, UR, gam, F);
  else hllc_y(UL, UR, gam, F);
}

/* HLL approximate Riemann solver in the x direction (Harten, Lax and van
   Leer 1983): the single intermediate state between S_L and S_R, with the
   wave speeds of hllc_x */
static void hll_x(const double* UL, const double* UR, double gam, double* F) {
  double rL = UL[0], uL = UL[1] / rL, vL = UL[2] / rL, EL = UL[3];
  double rR = UR[0], uR = UR[1] / rR, vR = UR[2] / rR, ER = UR[3];
  double pL = pressure(UL, gam), pR = pressure(UR, gam);
  double cL = sqrt(gam * pL / rL), cR = sqrt(gam * pR / rR);
  double SL = dmin2(uL - cL, uR - cR);
  double SR = dmax2(uL + cL, uR + cR);
  double FL[4] = {rL * uL, rL * uL * uL + pL, rL * uL * vL, uL * (EL + pL)};
  double FR[4] = {rR * uR, rR * uR * uR + pR, rR * uR * vR, uR * (ER + pR)};
  int dom = rL > 0.0 && rR > 0.0 && pL > 0.0 && pR > 0.0; /* else: flux undefined */
  for (int v = 0; v < 4; ++v) {
    if (!dom) F[v] = NAN;
    else if (SL >= 0.0) F[v] = FL[v];
    else if (SR > 0.0) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
    else F[v] = FR[v];
  }
}

static void hll_y(const double* UL, const double* UR, double gam, double* G) {
  double L[4] = {UL[0], UL[2], UL[1], UL[3]};
  double R[4] = {UR[0], UR[2], UR[1], UR[3]};
  double f[4];
  hll_x(L, R, gam, f);
  G[0] = f[0]; G[1] = f[2]; G[2] = f[1]; G[3] = f[3];
}

void orc_hll(const double* UL, const double* UR, double gam, int dir, double* F) {
  if (dir == 0) hll_x(UL, UR, gam, F);
  else hll_y(UL, UR, gam, F);
}

/* y-direction flux G by rotating (rho, rho v, rho u, E) through hllc_x */
static void hllc_y(const double* UL, const double* UR, double gam, double* G) {
  double L[4] = {UL[0], UL[2], UL[1], UL[3]};
  double R[4] = {UR[0], UR[2], UR[1], UR[3]};
  double f[4];
  hllc_x(L, R, gam, f);
  G[0] = f[0]; G[1] = f[2]; G[2] = f[1]; G[3] = f[3];
}

/* ------------------------------------------------------------------------- */
/* ghost cells                                                                */
/* ------------------------------------------------------------------------- */
static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

int orc_fill_ghosts(orc_ctx* c, const double* U, double t, double* Xg) {
  const orc_config* cf = &c->cfg;
  int nx = cf->nx, ny = cf->ny, H = c->H;
  double gam = cf->gamma;
  for (int v = 0; v < NV; ++v)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) Xg[gidx(c, v, i, j)] = U[iidx(c, v, i, j)];
  /* x pass: interior rows */
  for (int j = 0; j < ny; ++j)
    for (int k = 1; k <= H; ++k)
      for (int side = 0; side < 2; ++side) {
        int ig = side == 0 ? -k : nx - 1 + k;
        int kind = cf->bc[side];
        double S[4];
        if (kind == ORC_BC_DIRICHLET) {
          prim_to_cons(cf->bc_prim[side], gam, S);
        } else {
          int src;
          if (kind == ORC_BC_PERIODIC) src = wrap(ig, nx);
          else if (kind == ORC_BC_REFLECT) src = side == 0 ? k - 1 : nx - k;
          else src = side == 0 ? 0 : nx - 1;
          for (int v = 0; v < NV; ++v) S[v] = Xg[gidx(c, v, src, j)];
          if (kind == ORC_BC_REFLECT) S[1] = -S[1];
        }
        for (int v = 0; v < NV; ++v) Xg[gidx(c, v, ig, j)] = S[v];
      }
  /* y pass: every column including the x ghosts (fills the corners) */
  for (int i = -H; i < nx + H; ++i)
    for (int k = 1; k <= H; ++k)
      for (int side = 0; side < 2; ++side) {
        int jg = side == 0 ? -k : ny - 1 + k;
        double S[4];
        if (cf->dim == 1) {
          for (int v = 0; v < NV; ++v) S[v] = Xg[gidx(c, v, i, 0)];
        } else {
          int kind = cf->bc[2 + side];
          double xc = cf->x0 + (i + 0.5) * c->dx;
          int reflect = 0, fixed = 0;
          const double* P = 0;
          if (kind == ORC_BC_DIRICHLET) { fixed = 1; P = cf->bc_prim[2 + side]; }
          else if (kind == ORC_BC_DMR_BOTTOM) {
            if (xc < cf->dmr_wall_x0) { fixed = 1; P = cf->dmr_post; } else reflect = 1;
          } else if (kind == ORC_BC_DMR_TOP) {
            fixed = 1;
            P = (xc < cf->dmr_xs0 + cf->dmr_xs_speed * t) ? cf->dmr_post : cf->dmr_pre;
          } else if (kind == ORC_BC_JET) {
            /* jet_prim inside the slit, outflow elsewhere */
            if (xc >= cf->jet_x0 && xc <= cf->jet_x1) { fixed = 1; P = cf->jet_prim[side]; }
          } else if (kind == ORC_BC_REFLECT) reflect = 1;
          if (fixed) {
            prim_to_cons(P, gam, S);
          } else {
            int src;
            if (kind == ORC_BC_PERIODIC) src = wrap(jg, ny);
            else if (reflect) src = side == 0 ? k - 1 : ny - k;
            else src = side == 0 ? 0 : ny - 1;
            for (int v = 0; v < NV; ++v) S[v] = Xg[gidx(c, v, i, src)];
            if (reflect) S[2] = -S[2];
          }
        }
        for (int v = 0; v < NV; ++v) Xg[gidx(c, v, i, jg)] = S[v];
      }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* orders (Sec. 3.6 EDP1) and the cascade (Sec. 3.1 (iii))                    */
/* ------------------------------------------------------------------------- */
static int next_radius(const orc_ctx* c, int R) {
  for (int k = 0; k + 1 < c->cfg.ncascade; ++k)
    if (c->cfg.cascade[k] == R) return c->cfg.cascade[k + 1];
  return 0;
}

/* radius of a possibly-ghost cell: periodic ghosts carry the radius of the
   cell they copy; other ghosts carry the top radius, so a boundary face takes
   the radius of its interior cell under EDP1 */
static int radius_at(const orc_ctx* c, const uint8_t* ord, int i, int j) {
  const orc_config* cf = &c->cfg;
  if (i < 0 || i >= cf->nx) {
    if (cf->bc[0] != ORC_BC_PERIODIC) return c->top;
    i = wrap(i, cf->nx);
  }
  if (j < 0 || j >= cf->ny) {
    if (cf->dim == 1 || cf->bc[2] != ORC_BC_PERIODIC) return c->top;
    j = wrap(j, cf->ny);
  }
  return ord[(size_t)j * cf->nx + i];
}

/* face-state CAD flag for a possibly-ghost cell (periodic ghosts flag the
   cell they copy; other ghosts are not cells of the domain) */
static void mark_cad(orc_ctx* c, int i, int j) {
  const orc_config* cf = &c->cfg;
  if (i < 0 || i >= cf->nx) {
    if (cf->bc[0] != ORC_BC_PERIODIC) return;
    i = wrap(i, cf->nx);
  }
  if (j < 0 || j >= cf->ny) {
    if (cf->dim == 1 || cf->bc[2] != ORC_BC_PERIODIC) return;
    j = wrap(j, cf->ny);
  }
  c->cad[(size_t)j * cf->nx + i] = 1;
}

/* face-state check (Sec. 3.3.1, read with the Riemann solver's domain): a
   reconstructed state is admissible when its density and pressure are
   finite and positive -- the solver takes c = sqrt(gamma p / rho), which a
   non-positive p or rho leaves undefined */
static int finite_state(const double* U, double gam) {
  double p = pressure(U, gam);
  return isfinite(U[0]) && isfinite(p) && U[0] > 0.0 && p > 0.0;
}

/* reconstruct the pointwise state of cell (i,j) at Gauss point gi of face f
   with radius R (eq. gp_reconstructor; R = 0 is FOG, Sec. 2.6) */
static void reconstruct(const orc_ctx* c, const double* Xg, int R, int f, int gi, int i, int j,
                        double* Us) {
  if (R == 0) {
    for (int v = 0; v < NV; ++v) Us[v] = Xg[gidx(c, v, i, j)];
    return;
  }
  int n = c->n[R], q = c->q[R];
  if (c->cfg.poly3) {
    /* POL-MOOD3: p3 at the Gauss point of face f (Sec. 3.1 (iv)) */
    double xs, ys;
    qreal xq, yq;
    face_point(f, c->cfg.dim == 2 ? (qreal)c->gq[q][gi] : 0, &xq, &yq);
    xs = (double)xq;
    ys = (double)yq;
    for (int v = 0; v < NV; ++v) {
      double qv[MAXN];
      for (int m = 0; m < n; ++m)
        qv[m] = Xg[gidx(c, v, i + c->off[R][2 * m], j + c->off[R][2 * m + 1])];
      Us[v] = orc_poly3_eval(c->cfg.dim, qv, xs, ys);
    }
    return;
  }
  const double* z = c->z[R] + (size_t)(f * q + gi) * n;
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
    for (int m = 0; m < n; ++m) s += z[m] * Xg[gidx(c, v, i + c->off[R][2 * m], j + c->off[R][2 * m + 1])];
    Us[v] = s;
  }
}

/* x-face between cells (i-1,j) and (i,j): face-averaged flux by the Gauss rule
   of the face radius (eq. fvm_F), with face-state CAD (Sec. 3.3.1) */
static void face_flux_x(orc_ctx* c, const double* Xg, const uint8_t* ord, int i, int j) {
  int R = radius_at(c, ord, i - 1, j);
  int Rr = radius_at(c, ord, i, j);
  if (Rr < R) R = Rr; /* EDP1: the minimum of the two cells */
  int q = face_q(c->cfg.dim, R);
  double F[4] = {0, 0, 0, 0};
  for (int gi = 0; gi < q; ++gi) {
    double UL[4], UR[4], f[4];
    reconstruct(c, Xg, R, 0, gi, i - 1, j, UL); /* east face of the left cell */
    reconstruct(c, Xg, R, 1, gi, i, j, UR);     /* west face of the right cell */
    if (!finite_state(UL, c->cfg.gamma)) mark_cad(c, i - 1, j);
    if (!finite_state(UR, c->cfg.gamma)) mark_cad(c, i, j);
    if (c->cfg.riemann == 1) hll_x(UL, UR, c->cfg.gamma, f);
    else hllc_x(UL, UR, c->cfg.gamma, f);
    for (int v = 0; v < NV; ++v) F[v] += c->gw[q][gi] * f[v];
  }
  int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int v = 0; v < NV; ++v) c->Fx[((size_t)v * ny + j) * (nx + 1) + i] = F[v];
}

/* y-face between cells (i,j-1) and (i,j) */
static void face_flux_y(orc_ctx* c, const double* Xg, const uint8_t* ord, int i, int j) {
  int R = radius_at(c, ord, i, j - 1);
  int Rr = radius_at(c, ord, i, j);
  if (Rr < R) R = Rr;
  int q = face_q(c->cfg.dim, R);
  double G[4] = {0, 0, 0, 0};
  for (int gi = 0; gi < q; ++gi) {
    double UL[4], UR[4], f[4];
    reconstruct(c, Xg, R, 2, gi, i, j - 1, UL); /* north face of the lower cell */
    reconstruct(c, Xg, R, 3, gi, i, j, UR);     /* south face of the upper cell */
    if (!finite_state(UL, c->cfg.gamma)) mark_cad(c, i, j - 1);
    if (!finite_state(UR, c->cfg.gamma)) mark_cad(c, i, j);
    if (c->cfg.riemann == 1) hll_y(UL, UR, c->cfg.gamma, f);
    else hllc_y(UL, UR, c->cfg.gamma, f);
    for (int v = 0; v < NV; ++v) G[v] += c->gw[q][gi] * f[v];
  }
  int nx = c->cfg.nx;
  for (int v = 0; v < NV; ++v) c->Fy[((size_t)v * (c->cfg.ny + 1) + j) * nx + i] = G[v];
}

static void all_fluxes(orc_ctx* c, const double* Xg, const uint8_t* ord) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) face_flux_x(c, Xg, ord, i, j);
  if (c->cfg.dim == 2)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) face_flux_y(c, Xg, ord, i, j);
}

/* F_nabla of cell (i,j) (eq. fvm_F) from the stored face-averaged fluxes */
static void fnabla(const orc_ctx* c, int i, int j, double* Fn) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int v = 0; v < NV; ++v) {
    double fe = c->Fx[((size_t)v * ny + j) * (nx + 1) + i + 1];
    double fw = c->Fx[((size_t)v * ny + j) * (nx + 1) + i];
    double r = (fe - fw) / c->dx;
    if (c->cfg.dim == 2) {
      double gn = c->Fy[((size_t)v * (ny + 1) + j + 1) * nx + i];
      double gs = c->Fy[((size_t)v * (ny + 1) + j) * nx + i];
      r += (gn - gs) / c->dy;
    }
    Fn[v] = r;
  }
}

/* ------------------------------------------------------------------------- */
/* detection, Steps 4-9 of Sec. 4 (CAD, PAD, CSD, plateau, DMP, u2)           */
/* ------------------------------------------------------------------------- */
static double Xv(const orc_ctx* c, const double* Xg, int v, int i, int j) {
  return Xg[gidx(c, v, i, j)];
}

/* GP second derivative of the stage-input density at cell (i,j), App. B */
static double curvature(const orc_ctx* c, const double* Xg, int d, int i, int j) {
  int n = (c->cfg.dim == 2) ? 5 : 3;
  const double* w = d == 0 ? c->wxx : c->wyy;
  double s = 0.0;
  for (int m = 0; m < n; ++m) s += w[m] * Xv(c, Xg, 0, i + c->off1[2 * m], j + c->off1[2 * m + 1]);
  return s;
}

double orc_curvature(orc_ctx* c, const double* Xg, int d, int i, int j) {
  return curvature(c, Xg, d, i, j);
}

int orc_detect_cell(orc_ctx* c, const double* Xg, int i, int j, const double* Y4) {
  const orc_config* cf = &c->cfg;
  double gam = cf->gamma;
  int dim = cf->dim;
  double rho = Y4[0];
  double p = pressure(Y4, gam);
  /* Step 4, CAD (eq. CAD) */
  if (!isfinite(rho) || !isfinite(p)) return ORC_FAIL_CAD;
  /* Step 5, PAD (eq. PAD) */
  if (!(rho > 0.0) || !(p > 0.0)) return ORC_FAIL_PAD;
  /* Step 6, CSD (eqs. divV, gradP) on the stage input */
  if (cf->csd_on) {
    double uE = Xv(c, Xg, 1, i + 1, j) / Xv(c, Xg, 0, i + 1, j);
    double uW = Xv(c, Xg, 1, i - 1, j) / Xv(c, Xg, 0, i - 1, j);
    double pE, pW, pN, pS;
    double Sx[4], Sy[4];
    for (int v = 0; v < NV; ++v) { Sx[v] = Xv(c, Xg, v, i + 1, j); Sy[v] = Xv(c, Xg, v, i - 1, j); }
    pE = pressure(Sx, gam);
    pW = pressure(Sy, gam);
    double divV = (uE - uW) / (2.0 * c->dx);
    double gradP = fabs(pE - pW) / (2.0 * c->dx * dmin2(pE, pW));
    if (dim == 2) {
      double vN = Xv(c, Xg, 2, i, j + 1) / Xv(c, Xg, 0, i, j + 1);
      double vS = Xv(c, Xg, 2, i, j - 1) / Xv(c, Xg, 0, i, j - 1);
      for (int v = 0; v < NV; ++v) { Sx[v] = Xv(c, Xg, v, i, j + 1); Sy[v] = Xv(c, Xg, v, i, j - 1); }
      pN = pressure(Sx, gam);
      pS = pressure(Sy, gam);
      divV += (vN - vS) / (2.0 * c->dy);
      gradP += fabs(pN - pS) / (2.0 * c->dy * dmin2(pN, pS));
    }
    if (divV >= -cf->sigma_v && gradP <= cf->sigma_p) return ORC_ACCEPT_CSD;
  }
  /* neighbourhood {ij} U N(ij): the face neighbours */
  int nb = (dim == 2) ? 5 : 3;
  int ni[5] = {i, i - 1, i + 1, i, i};
  int nj[5] = {j, j, j, j + 1, j - 1};
  double rmin = Xv(c, Xg, 0, i, j), rmax = rmin;
  for (int m = 1; m < nb; ++m) {
    double r = Xv(c, Xg, 0, ni[m], nj[m]);
    rmin = dmin2(rmin, r);
    rmax = dmax2(rmax, r);
  }
  /* Step 7, plateau (eq. plateau) */
  double thr = c->dx * c->dx * c->dx;
  if (dim == 2) thr = dmin2(thr, c->dy * c->dy * c->dy);
  if (rmax - rmin < thr) return ORC_ACCEPT_PLATEAU;
  /* Step 8, DMP (eq. DMP_RK) */
  if (rmin <= rho && rho <= rmax) return ORC_ACCEPT_DMP;
  /* Step 9, u2 (eqs. u2_curvature, u2_a, u2_b), required for every direction */
  double delta = (dim == 2) ? dmin2(c->dx, c->dy) : c->dx;
  for (int d = 0; d < dim; ++d) {
    double cmin = curvature(c, Xg, d, ni[0], nj[0]), cmax = cmin;
    for (int m = 1; m < nb; ++m) {
      double k = curvature(c, Xg, d, ni[m], nj[m]);
      cmin = dmin2(cmin, k);
      cmax = dmax2(cmax, k);
    }
    int same_sign = cmin * cmax > -delta;
    int ua = same_sign && dmax2(fabs(cmax), fabs(cmin)) < delta;
    int ub = same_sign && fabs(cmin) / fabs(cmax) >= 0.5;
    if (!(ua || ub)) return ORC_FAIL_U2;
  }
  return ORC_ACCEPT_U2;
}

/* ------------------------------------------------------------------------- */
/* the spatial operator at fixed radii                                         */
/* ------------------------------------------------------------------------- */
int orc_residual(orc_ctx* c, const double* U, const uint8_t* ord, double t, double* Fn) {
  return orc_residual_cad(c, U, ord, t, Fn, 0);
}

/* the same, and (cad_out, nullable) the face-state check of every cell at
   these radii: 1 where a state its stencil produced on one of its faces
   failed (Sec. 3.3.1) */
int orc_residual_cad(orc_ctx* c, const double* U, const uint8_t* ord, double t, double* Fn,
                     uint8_t* cad_out) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  for (size_t k = 0; k < (size_t)nx * ny; ++k) {
    int R = ord[k];
    if (R != 0 && c->z[R] == 0) return -1;
  }
  orc_fill_ghosts(c, U, t, c->Xg);
  memset(c->cad, 0, (size_t)nx * ny);
  all_fluxes(c, c->Xg, ord);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double f[4];
      fnabla(c, i, j, f);
      for (int v = 0; v < NV; ++v) Fn[iidx(c, v, i, j)] = f[v];
    }
  if (cad_out) memcpy(cad_out, c->cad, (size_t)nx * ny);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* one MOOD stage (Sec. 4 Steps 3-10)                                          */
/* ------------------------------------------------------------------------- */
static void candidate_all(orc_ctx* c, const double* Xg, double dt, double* Y) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double f[4];
      fnabla(c, i, j, f);
      /* eq. fvm_discrete: forward-Euler sub-step of the RK stage */
      for (int v = 0; v < NV; ++v) Y[iidx(c, v, i, j)] = Xv(c, Xg, v, i, j) - dt * f[v];
    }
}

static int cell_troubled(orc_ctx* c, const double* Xg, const double* Y, int i, int j) {
  size_t k = (size_t)j * c->cfg.nx + i;
  if (c->ord[k] == 0) return 0; /* Step 10: FOG is accepted unchecked */
  if (c->cad[k]) return 1;
  double Y4[4];
  for (int v = 0; v < NV; ++v) Y4[v] = Y[iidx(c, v, i, j)];
  return orc_detect_cell(c, Xg, i, j, Y4) < 0;
}

/* neighbours of a cell for the MOOD update set (periodic wrap, no cell
   beyond a non-periodic boundary) */
static int cell_neighbours(const orc_ctx* c, int i, int j, int* ni, int* nj) {
  const orc_config* cf = &c->cfg;
  int n = 0;
  int cand_i[4] = {i - 1, i + 1, i, i};
  int cand_j[4] = {j, j, j - 1, j + 1};
  int nd = (cf->dim == 2) ? 4 : 2;
  for (int m = 0; m < nd; ++m) {
    int a = cand_i[m], b = cand_j[m];
    if (a < 0 || a >= cf->nx) {
      if (cf->bc[0] != ORC_BC_PERIODIC) continue;
      a = wrap(a, cf->nx);
    }
    if (b < 0 || b >= cf->ny) {
      if (cf->bc[2] != ORC_BC_PERIODIC) continue;
      b = wrap(b, cf->ny);
    }
    ni[n] = a; nj[n] = b; ++n;
  }
  return n;
}

/* one MOOD stage on the ghosted input Xg: the candidate Y = X - dt F(X) with
   the order cascade; Fn (nullable) receives the final F_nabla */
static int stage_on_ghosted(orc_ctx* c, const double* Xg, double dt, double* Y, int* iters_out,
                            int* nfirst_out, int* ntotal_out, double* Fn) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  size_t nc = (size_t)nx * ny;
  /* the highest order first, reset at every stage */
  memset(c->ord, c->top, nc);
  memset(c->cad, 0, nc);
  all_fluxes(c, Xg, c->ord);
  candidate_all(c, Xg, dt, Y);
  int nbad = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int b = cell_troubled(c, Xg, Y, i, j);
      c->bad[(size_t)j * nx + i] = (uint8_t)b;
      nbad += b;
    }
  if (nfirst_out) *nfirst_out = nbad;
  memcpy(c->first, c->bad, nc);
  int total = nbad, it = 0;
  while (nbad > 0) {
    if (it >= c->cfg.max_iters) return -3;
    ++it;
    /* the set whose candidates change: troubled cells and their neighbours */
    memset(c->inA, 0, nc);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (!c->bad[(size_t)j * nx + i]) continue;
        c->inA[(size_t)j * nx + i] = 1;
        int ni[4], nj[4];
        int n = cell_neighbours(c, i, j, ni, nj);
        for (int m = 0; m < n; ++m) c->inA[(size_t)nj[m] * nx + ni[m]] = 1;
      }
    /* order decrement by one cascade level */
    for (size_t k = 0; k < nc; ++k)
      if (c->bad[k]) c->ord[k] = (uint8_t)next_radius(c, c->ord[k]);
    memset(c->cad, 0, nc);
    all_fluxes(c, Xg, c->ord);
    candidate_all(c, Xg, dt, Y);
    nbad = 0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = (size_t)j * nx + i;
        int b = c->inA[k] ? cell_troubled(c, Xg, Y, i, j) : 0;
        c->bad[k] = (uint8_t)b;
        nbad += b;
      }
    total += nbad;
  }
  if (iters_out) *iters_out = it;
  if (ntotal_out) *ntotal_out = total;
  if (Fn)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double f[4];
        fnabla(c, i, j, f);
        for (int v = 0; v < NV; ++v) Fn[iidx(c, v, i, j)] = f[v];
      }
  return 0;
}

int orc_stage(orc_ctx* c, const double* X, double ts, double dt, double* Y, uint8_t* ord_out,
              uint8_t* bad_out, int* iters, int* nbad_total) {
  size_t nc = (size_t)c->cfg.nx * c->cfg.ny;
  orc_fill_ghosts(c, X, ts, c->Xg);
  int nfirst = 0;
  int rc = stage_on_ghosted(c, c->Xg, dt, Y, iters, &nfirst, nbad_total, 0);
  if (ord_out) memcpy(ord_out, c->ord, nc);
  if (bad_out) memcpy(bad_out, c->first, nc);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* time step (per-direction CFL form) and SSP-RK3 (eq. rk3)                    */
/* ------------------------------------------------------------------------- */
double orc_dt(orc_ctx* c, const double* U, double cfl) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  double gam = c->cfg.gamma, best = INFINITY;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double S[4];
      for (int v = 0; v < NV; ++v) S[v] = U[iidx(c, v, i, j)];
      double u = S[1] / S[0], v = S[2] / S[0];
      double cs = sqrt(gam * pressure(S, gam) / S[0]);
      double a = c->dx / (fabs(u) + cs);
      if (c->cfg.dim == 2) a = dmin2(a, c->dy / (fabs(v) + cs));
      if (!(a > 0.0) || !isfinite(a)) return NAN; /* no admissible step */
      best = dmin2(best, a);
    }
  /* the inflow state of a jet boundary enters the domain at the first step:
     its bound counts too (the quiescent ambient alone would give the jet a
     Courant number in the hundreds) */
  for (int side = 0; side < 2; ++side) {
    if (c->cfg.bc[2 + side] != ORC_BC_JET) continue;
    double S[4];
    prim_to_cons(c->cfg.jet_prim[side], gam, S);
    double u = S[1] / S[0], v = S[2] / S[0];
    double cs = sqrt(gam * pressure(S, gam) / S[0]);
    double a = dmin2(c->dx / (fabs(u) + cs), c->dy / (fabs(v) + cs));
    best = dmin2(best, a);
  }
  return cfl * best;
}

/* eq. rk4, the five-stage SSP-RK4, as printed:
     U^(s+1) = a_s U^n + b_s U^(s) - g_s Dt F(U^(s)),  s = 0..3, U^(0) = U^n,
     U^{n+1} = e2 U^(2) + e3 U^(3) - f3 Dt F(U^(3)) + e4 U^(4) - f4 Dt F(U^(4)).
   The printed final line carries "+ f3 Dt F(U^(3))"; every other Dt F term of
   the scheme enters with a minus and the weights of the Dt F terms must sum
   to one for consistency, so f3 is read with a minus (the stage times below
   then end at exactly one).  The MOOD candidate of a stage is its
   forward-Euler sub-step U^(s) - (g_s / b_s) Dt F(U^(s)), the same reading as
   for eq. rk3 (b_0 counts as one); the last stage's sub-step is
   U^(4) - (f4 / e4) Dt F(U^(4)).  Its U^(3) term, f3 / e3 = g_3 / b_3, is the
   sub-step already validated in stage 3. */
static const double RK4_A[4] = {1.0, 0.444370493651235, 0.620101851488403, 0.178079954393132};
static const double RK4_B[4] = {0.0, 0.555629506348765, 0.379898148511597, 0.821920045606868};
static const double RK4_G[4] = {0.391752226571890, 0.368410593050371, 0.251891774271694,
                                0.544974750228521};
static const double RK4_E2 = 0.517231671970585, RK4_E3 = 0.096059710526147,
                    RK4_F3 = 0.063692468666290, RK4_E4 = 0.386708617503269,
                    RK4_F4 = 0.226007483236906;

static int rk4_step(orc_ctx* c, double* U, double t, double dt, uint8_t* ord_out,
                    uint8_t* bad_out, orc_step_stats* st) {
  size_t nc = (size_t)c->cfg.nx * c->cfg.ny, ni = NV * nc;
  memcpy(c->U0, U, ni * sizeof(double));
  double* Us[5] = {c->U0, c->Us[1], c->Us[2], c->Us[3], c->Us[4]};
  double ts = 0.0; /* time of U^(s) as a fraction of Dt */
  for (int s = 0; s < 5; ++s) {
    double h = s < 4 ? RK4_G[s] / (s == 0 ? 1.0 : RK4_B[s]) : RK4_F4 / RK4_E4;
    orc_fill_ghosts(c, Us[s], t + ts * dt, c->Xg);
    int it = 0, nfirst = 0, ntot = 0;
    int rc = stage_on_ghosted(c, c->Xg, h * dt, c->Y, &it, &nfirst, &ntot, c->Fn);
    if (bad_out) memcpy(bad_out + s * nc, c->first, nc);
    if (ord_out) memcpy(ord_out + s * nc, c->ord, nc);
    if (st) {
      st->iters[s] = it;
      st->nbad_first[s] = nfirst;
      st->nbad_total[s] = ntot;
    }
    if (rc != 0) {
      if (st) st->status = rc;
      return rc;
    }
    if (s < 4) {
      for (size_t k = 0; k < ni; ++k)
        Us[s + 1][k] = RK4_A[s] * c->U0[k] + RK4_B[s] * Us[s][k] - RK4_G[s] * dt * c->Fn[k];
      if (s == 3) memcpy(c->F3, c->Fn, ni * sizeof(double));
      ts = RK4_B[s] * ts + RK4_G[s];
    } else {
      for (size_t k = 0; k < ni; ++k)
        U[k] = RK4_E2 * Us[2][k] + RK4_E3 * Us[3][k] - RK4_F3 * dt * c->F3[k] +
               RK4_E4 * Us[4][k] - RK4_F4 * dt * c->Fn[k];
    }
  }
  if (st) {
    st->dt = dt;
    st->status = 0;
  }
  return 0;
}

int orc_step(orc_ctx* c, double* U, double t, double cfl, double dt_fixed, uint8_t* ord_out,
             uint8_t* bad_out, orc_step_stats* st) {
  int nx = c->cfg.nx, ny = c->cfg.ny;
  size_t nc = (size_t)nx * ny, ni = NV * nc;
  double dt = dt_fixed > 0.0 ? dt_fixed : orc_dt(c, U, cfl);
  if (!(dt > 0.0) || !isfinite(dt)) {
    if (st) st->status = -4;
    return -4;
  }
  if (c->cfg.rk == 4) return rk4_step(c, U, t, dt, ord_out, bad_out, st);
  memcpy(c->U0, U, ni * sizeof(double));
  const double stage_t[3] = {t, t + dt, t + 0.5 * dt};
  for (int s = 0; s < 3; ++s) {
    /* stage input: U^n, U^(1), hat U^(2) */
    const double* Xin = (s == 0) ? c->U0 : c->S;
    orc_fill_ghosts(c, Xin, stage_t[s], c->Xg);
    int it = 0, nfirst = 0, ntot = 0;
    int rc = stage_on_ghosted(c, c->Xg, dt, c->Y, &it, &nfirst, &ntot, 0);
    if (bad_out) memcpy(bad_out + s * nc, c->first, nc);
    if (ord_out) memcpy(ord_out + s * nc, c->ord, nc);
    if (st) {
      st->iters[s] = it;
      st->nbad_first[s] = nfirst;
      st->nbad_total[s] = ntot;
    }
    if (rc != 0) {
      if (st) st->status = rc;
      return rc;
    }
    /* eq. rk3 */
    for (size_t k = 0; k < ni; ++k) {
      if (s == 0) c->S[k] = c->Y[k];
      else if (s == 1) c->S[k] = 0.25 * (3.0 * c->U0[k] + c->Y[k]);
      else U[k] = (c->U0[k] + 2.0 * c->Y[k]) / 3.0;
    }
  }
  if (st) {
    st->dt = dt;
    st->status = 0;
  }
  return 0;
}
