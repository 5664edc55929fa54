/*
 * gp_weights.c -- one-time GP weight solve on the host, in IEEE binary128.
 *
 * For a radius R the stencil is the blocky diamond |a| + |b| <= R (Sec. 2.2).
 * The volume-averaged SE covariance C (eq. SE-cov) and prediction kernel t*
 * (eq. SE-pred) factor over the two axes; the prediction vector is
 * z = C^{-1} t* (eq. gp_reconstructor), divided by its sum so that z^T 1 = 1
 * (eq. normalized_z, read as the signed sum).  The paper solves C in
 * quadruple precision and stores the result in double (Sec. 2.5); here the
 * symmetric positive-definite solve is an LDL^T factorisation (the
 * square-root-free form of Cholesky) in _Float128.
 *
 * Output order of the stencil: rows b = -R..R, and within a row a = -R..R,
 * keeping |a| + |b| <= R.
 *
 * Only the east and north faces at Gauss points g >= 0 are solved: the west
 * face is the x-mirror of the east face, the south face the y-mirror of the
 * north face, and the point -g the mirror of +g along the face, because the
 * kernel and the stencil are symmetric under both mirrors.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <string.h>

#include "gp_weights.h"

typedef _Float128 f128;

static f128 k_pi(void) { return 4 * atanf128(1); }

/* one axis of eq. SE-pred: mean over a unit cell of exp(-(s - d)^2 / (2 lam^2)) */
static f128 axis_pred(f128 d, f128 lam) {
  f128 h = sqrtf128(2) * lam;
  f128 hi = erff128((d + 0.5F128) / h);
  f128 lo = erff128((d - 0.5F128) / h);
  return lam * sqrtf128(k_pi() * 0.5F128) * (hi - lo);
}

/* G(u) = u erf(u) + exp(-u^2)/sqrt(pi); one axis of eq. SE-cov is
   sqrt(pi) lam^2 (G(u+) + G(u-) - 2 G(u0)) with u = (d+1, d-1, d)/(sqrt(2) lam) */
static f128 gfun(f128 u) { return u * erff128(u) + expf128(-u * u) / sqrtf128(k_pi()); }

static f128 axis_cov(f128 d, f128 lam) {
  f128 h = sqrtf128(2) * lam;
  f128 second_diff = gfun((d + 1) / h) + gfun((d - 1) / h) - 2 * gfun(d / h);
  return sqrtf128(k_pi()) * lam * lam * second_diff;
}

/* d^2/dx*^2 of one axis of eq. SE-pred, physical units (App. B) */
static f128 axis_pred_d2(f128 d, f128 lam, f128 ell) {
  f128 a = d - 0.5F128, b = d + 0.5F128;
  f128 two_l2 = 2 * lam * lam;
  return (a * expf128(-a * a / two_l2) - b * expf128(-b * b / two_l2)) / (ell * ell);
}

int gpw_stencil(int R, int* da, int* db) {
  int n = 0;
  for (int b = -R; b <= R; ++b)
    for (int a = -R; a <= R; ++a)
      if ((a < 0 ? -a : a) + (b < 0 ? -b : b) <= R) {
        da[n] = a;
        db[n] = b;
        ++n;
      }
  return n;
}

/* Table QR on [-1/2, 1/2]; points ordered from +1/2 to -1/2 */
static void gauss_q(int q, f128* gg, f128* ww) {
  if (q == 1) {
    gg[0] = 0; ww[0] = 1;
  } else if (q == 2) {
    gg[0] = 0.5F128 / sqrtf128(3); gg[1] = -gg[0];
    ww[0] = ww[1] = 0.5F128;
  } else if (q == 3) {
    gg[0] = 0.5F128 * sqrtf128(0.6F128); gg[1] = 0; gg[2] = -gg[0];
    ww[0] = ww[2] = 5.0F128 / 18; ww[1] = 8.0F128 / 18;
  } else {
    f128 r = (2.0F128 / 7) * sqrtf128(1.2F128);
    gg[0] = 0.5F128 * sqrtf128(3.0F128 / 7 + r);
    gg[1] = 0.5F128 * sqrtf128(3.0F128 / 7 - r);
    gg[2] = -gg[1]; gg[3] = -gg[0];
    ww[0] = ww[3] = (18 - sqrtf128(30)) / 72;
    ww[1] = ww[2] = (18 + sqrtf128(30)) / 72;
  }
}

void gpw_gauss(int q, double* g, double* w) {
  f128 gg[4], ww[4];
  gauss_q(q, gg, ww);
  for (int k = 0; k < q; ++k) {
    g[k] = (double)gg[k];
    w[k] = (double)ww[k];
  }
}

/* LDL^T of the n x n SPD matrix A (row-major), in place: unit-lower L below
   the diagonal and D on it.  Returns -1 if a pivot is not positive. */
static int ldlt(int n, f128* A) {
  for (int j = 0; j < n; ++j) {
    f128 d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k] * A[k * n + k];
    if (!(d > 0)) return -1;
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      f128 s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k] * A[k * n + k];
      A[i * n + j] = s / d;
    }
  }
  return 0;
}

static void ldlt_solve(int n, const f128* A, f128* x) {
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < i; ++k) x[i] -= A[i * n + k] * x[k];
  for (int i = 0; i < n; ++i) x[i] /= A[i * n + i];
  for (int i = n - 1; i >= 0; --i)
    for (int k = i + 1; k < n; ++k) x[i] -= A[k * n + i] * x[k];
}

#define MAXN 25

/* factor C for radius R with length scales lx = ell/dx, ly = ell/dy */
static int factor_cov(int R, f128 lx, f128 ly, int n, const int* da, const int* db, f128* A) {
  f128 cx[13], cy[13]; /* axis covariances for offsets -2R..2R */
  for (int d = -2 * R; d <= 2 * R; ++d) {
    cx[d + 2 * R] = axis_cov((f128)d, lx);
    cy[d + 2 * R] = axis_cov((f128)d, ly);
  }
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k)
      A[m * n + k] = cx[da[k] - da[m] + 2 * R] * cy[db[k] - db[m] + 2 * R];
  return ldlt(n, A);
}

int gpw_solve(int R, double dx, double dy, double ell, gpw_radius* out) {
  if (R < 1 || R > 3) return -1;
  memset(out, 0, sizeof(*out));
  int n = gpw_stencil(R, out->da, out->db);
  int q = R + 1;
  out->n = n;
  out->q = q;
  f128 lx = (f128)ell / (f128)dx, ly = (f128)ell / (f128)dy;
  f128 A[MAXN * MAXN];
  if (factor_cov(R, lx, ly, n, out->da, out->db, A) != 0) return -2;
  f128 gq[4], wq[4];
  gauss_q(q, gq, wq);
  for (int face = 0; face < 2; ++face) /* 0: east (x = +1/2), 1: north (y = +1/2) */
    for (int k = 0; k < q; ++k) {
      f128 gk = gq[k];
      f128 xs = face == 0 ? 0.5F128 : gk;
      f128 ys = face == 0 ? gk : 0.5F128;
      f128 z[MAXN];
      for (int m = 0; m < n; ++m)
        z[m] = axis_pred(xs - out->da[m], lx) * axis_pred(ys - out->db[m], ly);
      ldlt_solve(n, A, z);
      f128 sum = 0;
      for (int m = 0; m < n; ++m) sum += z[m];
      for (int m = 0; m < n; ++m) out->z[face][k][m] = (double)(z[m] / sum);
    }
  for (int k = 0; k < q; ++k) {
    out->g[k] = (double)gq[k];
    out->w[k] = (double)wq[k];
  }
  return 0;
}

int gpw_second_derivative(double dx, double dy, double ell, int* da, int* db, double* wxx,
                          double* wyy) {
  int n = gpw_stencil(1, da, db);
  f128 lx = (f128)ell / (f128)dx, ly = (f128)ell / (f128)dy, L = ell;
  f128 A[MAXN * MAXN];
  if (factor_cov(1, lx, ly, n, da, db, A) != 0) return -2;
  f128 tx[MAXN], ty[MAXN];
  for (int m = 0; m < n; ++m) {
    f128 ax = -(f128)da[m], ay = -(f128)db[m]; /* centre minus stencil point */
    tx[m] = axis_pred_d2(ax, lx, L) * axis_pred(ay, ly);
    ty[m] = axis_pred(ax, lx) * axis_pred_d2(ay, ly, L);
  }
  ldlt_solve(n, A, tx);
  ldlt_solve(n, A, ty);
  for (int m = 0; m < n; ++m) {
    wxx[m] = (double)tx[m];
    wyy[m] = (double)ty[m];
  }
  return n;
}

/* One-dimensional GP (dim = 1): the stencil a = -R..R, one face point at
   x = +1/2 (eq. SE-pred and eq. SE-cov with the x factor only), z divided by
   its sum.  The result is laid out as a 2D radius-R table so that the same
   kernels apply it: the weight of offset (a, 0) on the row b = 0, zero off
   that row, the same vector at each of the R+1 Gauss-point slots, and Gauss
   weights (1/2, 0, ..., 0, 1/2): every slot yields the same face state, and
   the first and last slots, a mirror pair of the kernels' pairwise Gauss
   sum, give exactly that state's flux. */
int gpw_solve_1d(int R, double dx, double ell, gpw_radius* out) {
  if (R < 1 || R > 3) return -1;
  memset(out, 0, sizeof(*out));
  int n = gpw_stencil(R, out->da, out->db);
  int q = R + 1;
  out->n = n;
  out->q = q;
  const int n1 = 2 * R + 1;
  f128 lx = (f128)ell / (f128)dx;
  f128 A[MAXN * MAXN];
  for (int m = 0; m < n1; ++m)
    for (int k = 0; k < n1; ++k) A[m * n1 + k] = axis_cov((f128)(k - m), lx);
  if (ldlt(n1, A) != 0) return -2;
  f128 z[MAXN];
  for (int m = 0; m < n1; ++m) z[m] = axis_pred(0.5F128 - (f128)(m - R), lx);
  ldlt_solve(n1, A, z);
  f128 sum = 0;
  for (int m = 0; m < n1; ++m) sum += z[m];
  for (int m = 0; m < n; ++m) {
    double zm = out->db[m] == 0 ? (double)(z[out->da[m] + R] / sum) : 0.0;
    for (int k = 0; k < q; ++k) out->z[0][k][m] = zm;
  }
  f128 gq[4], wq[4];
  gauss_q(q, gq, wq);
  for (int k = 0; k < q; ++k) {
    out->g[k] = (double)gq[k];
    out->w[k] = (k == 0 || k == q - 1) ? 0.5 : 0.0; /* q >= 2: a mirror pair of equal weight */
  }
  return 0;
}

/* App. B second-derivative weights of the one-dimensional GP on the
   3-point stencil, laid out on the 5-point R = 1 table (zero at (0, +-1));
   wyy is all zero */
int gpw_second_derivative_1d(double dx, double ell, int* da, int* db, double* wxx,
                             double* wyy) {
  int n = gpw_stencil(1, da, db);
  f128 lx = (f128)ell / (f128)dx, L = ell;
  f128 A[9], t[3];
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < 3; ++k) A[m * 3 + k] = axis_cov((f128)(k - m), lx);
  if (ldlt(3, A) != 0) return -2;
  for (int m = 0; m < 3; ++m) t[m] = axis_pred_d2(-(f128)(m - 1), lx, L);
  ldlt_solve(3, A, t);
  for (int m = 0; m < n; ++m) {
    wxx[m] = db[m] == 0 ? (double)t[da[m] + 1] : 0.0;
    wyy[m] = 0.0;
  }
  return n;
}

/* ------------------------------------------------------------------------- */
/* Poly3 of POL-MOOD3 (Sec. 3.1 (iv), eq. poly3 and eq. p3_coeffs): the       */
/* quadratic p = c0 + c1 x + c2 x^2 + c3 y + c4 y^2 whose means over the five  */
/* cells of the R = 1 stencil equal their cell averages.  The xy monomial has  */
/* zero mean on each of the five cells and cannot be fitted; it is left out.   */
/* With M[m][k] the mean of monomial k over stencil cell m, p(x*) =            */
/* phi(x*)^T M^{-1} qbar, so the weights at a point are z = M^{-T} phi(x*):   */
/* one small solve per point, in binary128 (cell units, origin at the centre). */
/* ------------------------------------------------------------------------- */

/* Gaussian elimination with partial pivoting on A x = b (n x n, row-major,
   both overwritten; x returned in b).  Returns -1 on a zero pivot. */
static int gesv(int n, f128* A, f128* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsf128(A[r * n + c]) > fabsf128(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        f128 t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
      }
      f128 t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      f128 f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    for (int k = r + 1; k < n; ++k) b[r] -= A[r * n + k] * b[k];
    b[r] /= A[r * n + r];
  }
  return 0;
}

/* the monomials 1, x, x^2, y, y^2 at a point, and their means over the unit
   cell centred at (a, b); nk = 3 keeps the x monomials only (1D) */
static void poly3_phi(f128 x, f128 y, f128* phi) {
  phi[0] = 1; phi[1] = x; phi[2] = x * x; phi[3] = y; phi[4] = y * y;
}
static void poly3_means(f128 a, f128 b, f128* mu) {
  const f128 v = 1.0F128 / 12; /* mean of s^2 over [-1/2, 1/2] */
  mu[0] = 1; mu[1] = a; mu[2] = a * a + v; mu[3] = b; mu[4] = b * b + v;
}

/* z = M^{-T} rhs over the stencil cells cell[0..nk-1] (offsets a, b) */
static int poly3_weights_at(int nk, const int* ca, const int* cb, const f128* rhs, f128* z) {
  f128 MT[25];
  for (int m = 0; m < nk; ++m) {
    f128 mu[5];
    poly3_means((f128)ca[m], (f128)cb[m], mu);
    for (int k = 0; k < nk; ++k) MT[k * nk + m] = mu[k]; /* row k = monomial k */
  }
  for (int k = 0; k < nk; ++k) z[k] = rhs[k];
  if (gesv(nk, MT, z) != 0) return -1;
  /* the exact weights are small rationals; where one is zero the elimination
     leaves binary128 round-off, which is cleared */
  f128 big = 0;
  for (int k = 0; k < nk; ++k) big = fabsf128(z[k]) > big ? fabsf128(z[k]) : big;
  for (int k = 0; k < nk; ++k)
    if (fabsf128(z[k]) < 1e-25F128 * big) z[k] = 0;
  return 0;
}

int gpw_poly3(gpw_radius* out) {
  memset(out, 0, sizeof(*out));
  int n = gpw_stencil(1, out->da, out->db);
  int q = 2; /* the two-point Gauss rule of the R = 1 faces */
  out->n = n;
  out->q = q;
  f128 gq[4], wq[4];
  gauss_q(q, gq, wq);
  for (int face = 0; face < 2; ++face)
    for (int k = 0; k < q; ++k) {
      f128 xs = face == 0 ? 0.5F128 : gq[k];
      f128 ys = face == 0 ? gq[k] : 0.5F128;
      f128 phi[5], z[5];
      poly3_phi(xs, ys, phi);
      if (poly3_weights_at(n, out->da, out->db, phi, z) != 0) return -2;
      for (int m = 0; m < n; ++m) out->z[face][k][m] = (double)z[m];
    }
  for (int k = 0; k < q; ++k) {
    out->g[k] = (double)gq[k];
    out->w[k] = (double)wq[k];
  }
  return 0;
}

/* 1D: the quadratic c0 + c1 x + c2 x^2 on the cells a = -1, 0, 1, laid out
   like gpw_solve_1d's R = 1 table (row b = 0, both Gauss slots the same
   vector, Gauss weights (1/2, 1/2)) */
int gpw_poly3_1d(gpw_radius* out) {
  memset(out, 0, sizeof(*out));
  int n = gpw_stencil(1, out->da, out->db);
  out->n = n;
  out->q = 2;
  const int ca[3] = {-1, 0, 1}, cb[3] = {0, 0, 0};
  f128 phi[5], z[5];
  poly3_phi(0.5F128, 0, phi);
  if (poly3_weights_at(3, ca, cb, phi, z) != 0) return -2;
  for (int m = 0; m < n; ++m) {
    double zm = out->db[m] == 0 ? (double)z[out->da[m] + 1] : 0.0;
    out->z[0][0][m] = out->z[0][1][m] = zm;
  }
  f128 gq[4], wq[4];
  gauss_q(2, gq, wq);
  for (int k = 0; k < 2; ++k) {
    out->g[k] = (double)gq[k];
    out->w[k] = 0.5;
  }
  return 0;
}

/* u2 curvatures of POL-MOOD3 (eq. u2_curvature): the second derivatives of
   Poly3 at the cell centre, d^2 p / dx^2 = 2 c2 and d^2 p / dy^2 = 2 c4, in
   physical units, as weights z = M^{-T} phi'' on the 5-point R = 1 table;
   one_d: the 3-cell fit, wyy zero */
int gpw_second_derivative_poly3(int one_d, double dx, double dy, int* da, int* db,
                                double* wxx, double* wyy) {
  int n = gpw_stencil(1, da, db);
  f128 rx[5] = {0, 0, 2, 0, 0}, ry[5] = {0, 0, 0, 0, 2}, zx[5], zy[5];
  if (one_d) {
    const int ca[3] = {-1, 0, 1}, cb[3] = {0, 0, 0};
    if (poly3_weights_at(3, ca, cb, rx, zx) != 0) return -2;
    for (int m = 0; m < n; ++m) {
      wxx[m] = db[m] == 0 ? (double)(zx[da[m] + 1] / ((f128)dx * dx)) : 0.0;
      wyy[m] = 0.0;
    }
    return n;
  }
  if (poly3_weights_at(n, da, db, rx, zx) != 0) return -2;
  if (poly3_weights_at(n, da, db, ry, zy) != 0) return -2;
  for (int m = 0; m < n; ++m) {
    wxx[m] = (double)(zx[m] / ((f128)dx * dx));
    wyy[m] = (double)(zy[m] / ((f128)dy * dy));
  }
  return n;
}
