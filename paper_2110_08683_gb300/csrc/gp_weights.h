/* gp_weights.h -- host-side binary128 GP weight solve (see gp_weights.c). */
#ifndef GPMOOD_GP_WEIGHTS_H
#define GPMOOD_GP_WEIGHTS_H
#ifdef __cplusplus
extern "C" {
#endif

/* prediction vectors of one radius: z[face][k][m], face 0 = east, 1 = north,
   k over the q Gauss points g[k] (ordered +1/2 .. -1/2), m over the stencil
   (da[m], db[m]) */
typedef struct {
  int n, q;
  int da[25], db[25];
  double g[4], w[4];
  double z[2][4][25];
} gpw_radius;

int gpw_stencil(int R, int* da, int* db);
void gpw_gauss(int q, double* g, double* w);
/* returns 0, -1 for a bad radius, -2 if C is not positive definite */
int gpw_solve(int R, double dx, double dy, double ell, gpw_radius* out);
/* App. B second-derivative weights on the R = 1 stencil, physical units;
   returns the stencil size (5) or -2 */
int gpw_second_derivative(double dx, double dy, double ell, int* da, int* db, double* wxx,
                          double* wyy);
/* the one-dimensional GP (stencil a = -R..R, one face point) laid out as a
   2D radius-R table: weights on the row b = 0, the same vector at every
   Gauss-point slot, Gauss weights (1/2, 0, ..., 0, 1/2); north-face weights zero */
int gpw_solve_1d(int R, double dx, double ell, gpw_radius* out);
/* the 1D App. B second-derivative weights on the 5-point table (wyy = 0) */
int gpw_second_derivative_1d(double dx, double ell, int* da, int* db, double* wxx,
                             double* wyy);

/* POL-MOOD3 (Sec. 3.1 (iv)): Poly3, the quadratic of eq. poly3 fitted to the
   five cell averages of the R = 1 stencil (eq. p3_coeffs), evaluated at the
   face Gauss points; the same layout as gpw_solve(1, ...).  Returns 0 or -2 */
int gpw_poly3(gpw_radius* out);
/* the 1D Poly3 (three cells) laid out like gpw_solve_1d(1, ...) */
int gpw_poly3_1d(gpw_radius* out);
/* POL-MOOD3's u2 curvature weights: Poly3's second derivatives at the cell
   centre, physical units, on the 5-point table; returns 5 or -2 */
int gpw_second_derivative_poly3(int one_d, double dx, double dy, int* da, int* db,
                                double* wxx, double* wyy);

#ifdef __cplusplus
}
#endif
#endif
