/*
 * gpmood_oracle.h -- plain, slow FP64 CPU oracle of GP-MOOD (Bourgeois & Lee,
 * "GP-MOOD: A positive-preserving high-order finite volume method for
 * hyperbolic conservation laws", arXiv:2110.08683).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  It
 * shares no code with it (no headers, helpers, tables or constant generators)
 * and must only be loaded by the test suite, the smoke check and the CPU
 * baseline leg of the benchmark.  The product path never calls it.
 *
 * Everything is FP64 except the one-time GP weight solve, which is done in
 * IEEE binary128 (_Float128) as the paper prescribes (Sec. 2.5) and rounded
 * to double.  Loops are written in the order of the paper's definitions with
 * no blocking or fusion.
 *
 * Array layout: conservative variables U = (rho, rho u, rho v, rho E) are
 * stored structure-of-arrays, variable-major, row-major within a variable:
 *   interior arrays  U[v][j][i]            v<4, j<ny, i<nx
 *   ghosted arrays   X[v][j+H][i+H]        with H ghost layers on each side
 */
#ifndef GPMOOD_ORACLE_H
#define GPMOOD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* boundary condition kinds, per side (W, E, S, N) */
enum {
  ORC_BC_PERIODIC = 0,
  ORC_BC_OUTFLOW = 1,    /* zero gradient: ghost copies the nearest interior cell */
  ORC_BC_REFLECT = 2,    /* mirror, normal momentum negated */
  ORC_BC_DIRICHLET = 3,  /* fixed primitive state bc_prim[side] */
  ORC_BC_DMR_BOTTOM = 4, /* S side: x < wall_x0 -> state post, else reflect */
  ORC_BC_DMR_TOP = 5,    /* N side: x < xs0 + xs_speed*t -> post, else pre */
  ORC_BC_JET = 6         /* S or N side: jet_prim inside jet_x0 <= x <= jet_x1 (cell
                            centres), outflow elsewhere (Sec. 5.3, the Mach jets) */
};

/* detection outcome codes for a single cell (Steps 4-9 of Sec. 4) */
enum {
  ORC_ACCEPT_CSD = 1,
  ORC_ACCEPT_PLATEAU = 2,
  ORC_ACCEPT_DMP = 3,
  ORC_ACCEPT_U2 = 4,
  ORC_FAIL_CAD = -1,
  ORC_FAIL_PAD = -2,
  ORC_FAIL_U2 = -3
};

typedef struct {
  int dim;               /* 1 or 2 */
  int nx, ny;            /* interior cells (ny = 1 when dim = 1) */
  double x0, x1, y0, y1; /* domain */
  int bc[4];             /* W, E, S, N */
  double bc_prim[4][4];  /* Dirichlet primitive state (rho,u,v,p) per side */
  double gamma;
  int ncascade;          /* number of entries in cascade[] */
  int cascade[4];        /* GP radii, strictly decreasing, last entry 0 (FOG) */
  double ell;            /* SE length scale, physical units */
  double sigma_v, sigma_p;
  int csd_on;
  int max_iters;         /* MOOD iteration cap per stage */
  /* double Mach reflection boundary data (used by the DMR_* kinds) */
  double dmr_post[4], dmr_pre[4];
  double dmr_wall_x0, dmr_xs0, dmr_xs_speed;
  int rk;                /* 3 (or 0): SSP-RK3, eq. rk3; 4: five-stage SSP-RK4, eq. rk4 */
  int riemann;           /* 0: HLLC (Toro et al. 1994); 1: HLL (Harten, Lax, van Leer 1983) */
  double jet_x0, jet_x1; /* inflow slit of the JET kind */
  double jet_prim[2][4]; /* jet state (rho, u, v, p) on the S and N sides */
  int poly3;             /* 1: POL-MOOD3 (Sec. 3.1 (iv)): the R = 1 rung is Poly3
                            (eq. poly3, App. C) instead of GP-R1, and the u2 curvatures
                            are the second derivatives of p3; cascade must be {1, 0} */
} orc_config;

typedef struct orc_ctx orc_ctx;

/* per-step diagnostics */
typedef struct {
  double dt;
  int iters[5];          /* MOOD iterations per RK stage (0 = first pass clean) */
  int nbad_first[5];     /* troubled cells after the first pass, per stage */
  int nbad_total[5];     /* sum over iterations of troubled-cell counts */
  int status;            /* 0 ok, <0 error */
} orc_step_stats;       /* the first 3 (RK3) or 5 (RK4) entries are used */

int orc_create(const orc_config* cfg, orc_ctx** out);
void orc_destroy(orc_ctx* ctx);
int orc_ghost_width(const orc_ctx* ctx);

/* --- GP building blocks (Sec. 2.3-2.5, App. A-B) --- */
/* stencil of radius R: fills off[2*N] with (a,b) offsets, returns N */
int orc_stencil(int dim, int R, int* off);
/* Gauss-Legendre rule on [-1/2,1/2] (Table "QR"), q = 1..4 */
int orc_gauss_rule(int q, double* g, double* w);
/* volume-averaged kernels eq. SE-pred and SE-cov in one dimension (cell units) */
double orc_pred_1d(double delta, double lam);
double orc_cov_1d(double delta, double lam);
/* prediction vectors z[face][g][m] for radius R, faces E,W,N,S (dim=1: E,W), normalised */
int orc_gp_weights(int dim, int R, double lamx, double lamy, double* z, int* nq, int* nn);
/* the same before the normalisation eq. normalized_z */
int orc_gp_weights_raw(int dim, int R, double lamx, double lamy, double* z);
/* App. B second-derivative weights at the cell centre on the R=1 stencil */
int orc_d2_weights(int dim, double ell, double dx, double dy, double* wxx, double* wyy);
/* Poly3 (eq. poly3 with the App. C coefficients) of the cell whose R = 1
   stencil values, in orc_stencil order, are qv, evaluated at (xs, ys) in cell
   units from the cell centre; dim 1 reads the data as constant in y */
double orc_poly3_eval(int dim, const double* qv, double xs, double ys);

/* --- scheme --- */
/* HLLC flux between pointwise states UL, UR across an x (dir 0) or y (dir 1) face */
void orc_hllc(const double* UL, const double* UR, double gamma, int dir, double* F);
/* HLL flux with the same wave speeds */
void orc_hll(const double* UL, const double* UR, double gamma, int dir, double* F);
/* F_nabla (eq. fvm_F) of the interior state U at per-cell radii ord (EDP1 faces) */
int orc_residual(orc_ctx* ctx, const double* U, const uint8_t* ord, double t, double* Fn);
int orc_residual_cad(orc_ctx* ctx, const double* U, const uint8_t* ord, double t, double* Fn,
                     uint8_t* cad_out);
/* Delta t from U (per-direction CFL form) */
double orc_dt(orc_ctx* ctx, const double* U, double cfl);
/* one SSP-RK3 (or SSP-RK4, cfg.rk = 4) step with the MOOD loop; dt_fixed > 0
   overrides the CFL step.  ord_out (nullable) receives [S][ny][nx] final radii
   per stage, bad_out (nullable) the [S][ny][nx] first-pass troubled-cell map,
   S = 3 (RK3) or 5 (RK4). */
int orc_step(orc_ctx* ctx, double* U, double t, double cfl, double dt_fixed,
             uint8_t* ord_out, uint8_t* bad_out, orc_step_stats* st);
/* one MOOD stage: candidate Y = X - dt F(X) with the order cascade, from the
   interior stage input X at time ts.  ord_out [ny][nx], bad_out [ny][nx]. */
int orc_stage(orc_ctx* ctx, const double* X, double ts, double dt, double* Y,
              uint8_t* ord_out, uint8_t* bad_out, int* iters, int* nbad_total);
/* detection of one cell (Steps 4-9) given the ghosted stage input X and the
   candidate Y4 of that cell; returns an ORC_ACCEPT_* or ORC_FAIL_* code */
int orc_detect_cell(orc_ctx* ctx, const double* Xg, int i, int j, const double* Y4);
/* the u2 curvature (eq. u2_curvature) of the density of ghosted state Xg at
   interior cell (i, j) along direction d (0: x, 1: y), physical units */
double orc_curvature(orc_ctx* ctx, const double* Xg, int d, int i, int j);
/* ghost fill of an interior array into a ghosted array at time t */
int orc_fill_ghosts(orc_ctx* ctx, const double* U, double t, double* Xg);

#ifdef __cplusplus
}
#endif
#endif
