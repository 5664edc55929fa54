// gpmood_kernels.cuh -- CUDA kernels of the GP-MOOD stage (sm_103a).
//
// One RK stage (Sec. 4, Steps 3-10) of a single problem runs as
//   fill_ghosts -> x_faces -> y_faces -> update_first    (first pass, all cells)
//   mood_loop                                             (troubled cells only)
// x_faces / y_faces reconstruct the pointwise Riemann states of eq.
// gp_reconstructor at the Gauss points of Table QR, apply face-state CAD
// (Sec. 3.3.1), solve HLLC and store the face-averaged flux of eq. fvm_F.
// update_first forms the candidate of eq. fvm_discrete, runs Steps 4-9,
// writes the SSP-RK3 combination (eq. rk3) and appends troubled cells to a
// queue with one atomic per warp.  mood_loop iterates on the device, with
// grid-wide barriers between its phases: it lowers the order of queued cells
// by one cascade level, recomputes the faces whose EDP1 order changed (Sec.
// 3.6) and re-updates + re-detects the queued cells and their face
// neighbours, until no cell is troubled.  Batches run the same phases as one
// kernel per phase, the loop a conditional WHILE node of the step graph.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gpmood_internal.h"
#include "fp_bits.h"

namespace gpm {

// ---------------------------------------------------------------------------
// indexing
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long gidx(const Grid& g, int v, int i, int j) {
  return (long long)v * g.vstride + (long long)(j + g.H) * g.pitch + (i + g.H);
}
// x-face i (0..nx) of row j: between cells i-1 and i
__device__ __forceinline__ long long fxidx(const Grid& g, int v, int i, int j) {
  return ((long long)v * g.ny + j) * (g.nx + 1) + i;
}
// y-face j (0..ny) of column i: between cells j-1 and j
__device__ __forceinline__ long long fyidx(const Grid& g, int v, int i, int j) {
  return ((long long)v * (g.ny + 1) + j) * g.nx + i;
}
__device__ __forceinline__ int cidx(const Grid& g, int i, int j) { return j * g.nx + i; }

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// stencil algebra at compile time.
// The blocky diamond |a|+|b| <= R is invariant under x -> -x and y -> -y, and
// so is the SE kernel; hence the west-face weights are the x-mirror of the
// east-face ones, the point -g the mirror of +g, and the same for north /
// south.  Grouping the stencil into mirror orbits {(+-a, +-b)} and using the
// even/odd combinations of each orbit ("parity sums") turns the 2q face
// states of one axis into q dot products of length N plus butterflies,
// instead of 2q dot products.  The parity sums of one cell are shared by all
// four faces.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int stencil_n(int R) { return 2 * R * R + 2 * R + 1; }
__host__ __device__ constexpr int rule_q(int R) { return R == 0 ? 1 : R + 1; }

struct Comp {
  int a, b, px, py;
};

// k-th parity component: reps (a,b) with a,b >= 0, a+b <= R in order b-major,
// and for each rep the types ee, oe (a>0), eo (b>0), oo (a,b>0)
__host__ __device__ constexpr Comp comp_at(int R, int k) {
  int n = 0;
  for (int b = 0; b <= R; ++b)
    for (int a = 0; a + b <= R; ++a) {
      if (n == k) return Comp{a, b, 0, 0};
      ++n;
      if (a > 0) {
        if (n == k) return Comp{a, b, 1, 0};
        ++n;
      }
      if (b > 0) {
        if (n == k) return Comp{a, b, 0, 1};
        ++n;
      }
      if (a > 0 && b > 0) {
        if (n == k) return Comp{a, b, 1, 1};
        ++n;
      }
    }
  return Comp{0, 0, 0, 0};
}

// parity sums of one variable around a cell; ld(a, b) loads the cell (i+a, j+b)
template <int R, class Real, class Load>
__device__ __forceinline__ void parity_sums(const Load& ld, Real* s) {
  int k = 0;
#pragma unroll
  for (int b = 0; b <= R; ++b) {
#pragma unroll
    for (int a = 0; a + b <= R; ++a) {
      if (a == 0 && b == 0) {
        s[k++] = ld(0, 0);
      } else if (b == 0) {
        Real p = ld(a, 0), m = ld(-a, 0);
        s[k++] = p + m;
        s[k++] = p - m;
      } else if (a == 0) {
        Real p = ld(0, b), m = ld(0, -b);
        s[k++] = p + m;
        s[k++] = p - m;
      } else {
        Real q1 = ld(a, b), q2 = ld(-a, b), q3 = ld(a, -b), q4 = ld(-a, -b);
        Real p1 = q1 + q2, m1 = q1 - q2, p2 = q3 + q4, m2 = q3 - q4;
        s[k++] = p1 + p2;  // ee
        s[k++] = m1 + m2;  // oe
        s[k++] = p1 - p2;  // eo
        s[k++] = m1 - m2;  // oo
      }
    }
  }
}

// T[px][py] = sum over components of that parity of c[k] s[k]
template <int R, class Real>
__device__ __forceinline__ void parity_dot(const Real* c, const Real* s, Real T[2][2]) {
  T[0][0] = T[0][1] = T[1][0] = T[1][1] = Real(0);
#pragma unroll
  for (int k = 0; k < stencil_n(R); ++k) {
    const Comp cm = comp_at(R, k);
    T[cm.px][cm.py] = fma(c[k], s[k], T[cm.px][cm.py]);
  }
}

// ---------------------------------------------------------------------------
// Euler equations (eq. euler_eqn) and HLLC (Toro et al. 1994) in Real
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ Real pressure_of(const Real* U, Real gm1) {
  Real ir = Real(1) / U[0];
  return gm1 * (U[3] - Real(0.5) * (U[1] * U[1] + U[2] * U[2]) * ir);
}

// finite (neither infinite nor NaN), decided on the bit pattern
__device__ __forceinline__ bool finite_r(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffll) < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }

// reciprocal from the hardware approximation r (rcp.approx.ftz.f64, whose
// relative error stays below 2^-20 on this GPU): with e = 1 - x r,
// 1/x = r / (1 - e) = r (1 + e + e^2 + ...), and the series cut after e^2
// leaves a relative error below 2^-60 before the final rounding (one FMA
// fewer than two Newton-Raphson steps).  FP32: rcp.approx.ftz.f32 (within 1
// ulp) and one Newton-Raphson step r + r (1 - x r).  Zero or non-finite x
// give a non-finite result.
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// square root of a sound-speed argument z > 0 (the Riemann solvers; outside
// their domain the result is NaN, and so is their flux).  FP64: from the
// hardware inverse square root y (rsqrt.approx.ftz.f64, relative error below
// 2^-20 on this GPU), s = z y and two corrections s <- s + (y/2)(z - s^2),
// each of which multiplies the relative error by about that of y: within
// one unit in the last place, in six FP64 operations where the IEEE square
// root takes the FP64 pipe about as long as seven and a half.  FP32: the
// hardware approximation sqrt.approx.ftz.f32 (the FP32 path's reconstruction
// and Riemann solver are FP32 arithmetic throughout).
__device__ __forceinline__ double sqrt_r(double z) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(z));
  const double h = __dmul_rn(0.5, y);
  double s = __dmul_rn(z, y);
  s = fma(h, fma(-s, s, z), s);
  return fma(h, fma(-s, s, z), s);
}
__device__ __forceinline__ float sqrt_r(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// products and sums rounded one by one (no contraction into an FMA): where
// an expression's mirror image swaps its terms, both then round alike, so a
// mirror-symmetric problem stays symmetric bit for bit
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// pressure of a conservative state with 1/rho given, the velocities out: one
// fixed sequence of rounded operations, so two states that are mirror images
// (a momentum component negated) give the same pressure bit for bit, whichever
// side of a face or of a cell each sits on
template <class Real>
__device__ __forceinline__ Real pressure_ir(const Real* U, Real ir, Real gm1, Real& u, Real& v) {
  u = mul_rn(U[1], ir);
  v = mul_rn(U[2], ir);
  const Real k = fma(U[1], u, mul_rn(U[2], v));  // m_x u + m_y v
  return mul_rn(gm1, fma(Real(-0.5), k, U[3]));
}

// quiet NaN: the flux of a face whose state lies outside the Riemann solver's
// domain (non-positive or non-finite density or pressure) is undefined
__device__ __forceinline__ void qnan(double& x) { x = __longlong_as_double(0x7ff8000000000000ll); }
__device__ __forceinline__ void qnan(float& x) { x = __int_as_float(0x7fc00000); }
// x > 0 and finite, decided on the integer bits (positive finite values are
// the bit patterns strictly between +0 and +inf; NaN and negatives fall
// outside): the same answer as the two comparisons without denormal
// flushing, taken off the floating-point pipes
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool pos_finite(float x) {
  const int b = __float_as_int(x);
  return b > 0 && b < 0x7f800000;
}
// comparisons of doubles on the integer pipes (fp_bits.h: the IEEE answer
// exactly, for the inputs each name allows).  An FP64 compare, min or max
// occupies the FP64 pipe like an FMA does (on this GPU about 64 cycles per
// warp instruction per sub-partition), a 64-bit integer compare a few
// cycles.  FP32 keeps the hardware compare, which is cheap.
__device__ __forceinline__ bool is_nan(double x) { return fpb_is_nan(x); }
// a < b, a and b not NaN
__device__ __forceinline__ bool lt_num(double a, double b) { return fpb_lt_num(a, b); }
__device__ __forceinline__ bool lt_num(float a, float b) { return a < b; }
// a < b with NaN (false when either is NaN)
__device__ __forceinline__ bool lt_ieee(double a, double b) { return fpb_lt_ieee(a, b); }
__device__ __forceinline__ bool lt_ieee(float a, float b) { return a < b; }
// a <= b with NaN (false when either is NaN)
__device__ __forceinline__ bool le_ieee(double a, double b) { return fpb_le_ieee(a, b); }
__device__ __forceinline__ bool le_ieee(float a, float b) { return a <= b; }
// x >= 0 and x > 0, x not NaN
__device__ __forceinline__ bool ge0_num(double x) { return fpb_ge0_num(x); }
__device__ __forceinline__ bool ge0_num(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool gt0_num(double x) { return fpb_gt0_num(x); }
__device__ __forceinline__ bool gt0_num(float x) { return x > 0.0f; }
// a < b ? a : b and a > b ? a : b, a and b not NaN
template <class Real>
__device__ __forceinline__ Real min_num(Real a, Real b) { return lt_num(a, b) ? a : b; }
template <class Real>
__device__ __forceinline__ Real max_num(Real a, Real b) { return lt_num(b, a) ? a : b; }

template <class Real>
__device__ __forceinline__ bool solver_domain(Real rL, Real rR, Real pL, Real pR) {
  // rho > 0 and p > 0 (non-finite inputs give a NaN flux anyway)
  return pos_finite(rL) && pos_finite(rR) && pos_finite(pL) && pos_finite(pR);
}

// x-direction HLLC flux; pL/pR return the pressures of the two states so the
// caller can run face-state CAD without another EoS evaluation.
// wave speeds S_L = min(uL-cL, uR-cR), S_R = max(uL+cL, uR+cR); the star
// state is taken on the side of the contact speed S*.  Every product is an
// explicit fma or a product rounded on its own, so the compiler cannot fuse
// operations differently in different kernels: every kernel that solves a
// face gets the same flux bit for bit.  Inside the solver's domain every
// value is finite, so the comparisons run on the integer pipes (outside it
// the flux is NaN whatever they decide).
template <class Real>
__device__ __forceinline__ void hllc_x(const Real* UL, const Real* UR, Real gam, Real* F,
                                       Real& pL, Real& pR) {
  const Real gm1 = gam - Real(1);
  Real rL = UL[0], rR = UR[0];
  Real irL = recip(rL), irR = recip(rR);
  Real uL, vL, uR, vR;
  pL = pressure_ir(UL, irL, gm1, uL, vL);
  pR = pressure_ir(UR, irR, gm1, uR, vR);
  Real cL = sqrt_r(mul_rn(mul_rn(gam, pL), irL)), cR = sqrt_r(mul_rn(mul_rn(gam, pR), irR));
  const Real SL = min_num(uL - cL, uR - cR);
  const Real SR = max_num(uL + cL, uR + cR);
  Real dL = SL - uL, dR = SR - uR;
  const Real mL = mul_rn(rL, uL), mR = mul_rn(rR, uR);
  Real num = fma(-mR, dR, fma(mL, dL, pR - pL));
  Real den = fma(-rR, dR, mul_rn(rL, dL));
  Real Ss = mul_rn(num, recip(den));
  const bool left = ge0_num(Ss);
  const bool useL = ge0_num(SL);
  const bool useS = left || gt0_num(SR);
  // star state on side K of the contact: with m = rho_K (S_K - u_K) and
  // D = 1 / (S_K - S*), rho* = m D and
  //   (rho E)* = rho* (E_K/rho_K + (S* - u_K)(S* + p_K / m))
  //            = D ((S_K - u_K) E_K + (S* - u_K)(m S* + p_K)),
  // the second form needing no reciprocal of rho_K (S_K - u_K)
  Real rK = left ? rL : rR, uK = left ? uL : uR, vK = left ? vL : vR;
  Real EK = left ? UL[3] : UR[3], pK = left ? pL : pR, SK = left ? SL : SR;
  Real dK = left ? dL : dR;
  const Real m = mul_rn(rK, dK), iD = recip(SK - Ss);
  Real fK = mul_rn(m, iD);
  Real UKs[4] = {fK, mul_rn(fK, Ss), mul_rn(fK, vK),
                 mul_rn(iD, fma(dK, EK, mul_rn(Ss - uK, fma(m, Ss, pK))))};
  // one physical flux is ever used: F_L when S_L >= 0, F_R when S_R <= 0,
  // else the star flux F_K + S_K (U*_K - U_K) on side K
  const bool sideL = useL || (useS && left);
  const Real uX = sideL ? uL : uR, vX = sideL ? vL : vR, pX = sideL ? pL : pR;
  const Real mX = sideL ? mL : mR, EX = sideL ? UL[3] : UR[3];
  const Real FX[4] = {mX, fma(mX, uX, pX), mul_rn(mX, vX), mul_rn(uX, EX + pX)};
  const bool star = !useL && useS;
  const bool dom = solver_domain(rL, rR, pL, pR);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const Real UK = left ? UL[v] : UR[v];
    F[v] = star ? fma(SK, UKs[v] - UK, FX[v]) : FX[v];
    if (!dom) qnan(F[v]);
  }
}

// x-direction HLL flux (Harten, Lax and van Leer 1983): the single
// intermediate state between the wave speeds of hllc_x; pL/pR as there
template <class Real>
__device__ __forceinline__ void hll_x(const Real* UL, const Real* UR, Real gam, Real* F,
                                      Real& pL, Real& pR) {
  const Real gm1 = gam - Real(1);
  Real rL = UL[0], rR = UR[0];
  Real irL = recip(rL), irR = recip(rR);
  Real uL, vL, uR, vR;
  pL = pressure_ir(UL, irL, gm1, uL, vL);
  pR = pressure_ir(UR, irR, gm1, uR, vR);
  Real cL = sqrt_r(mul_rn(mul_rn(gam, pL), irL)), cR = sqrt_r(mul_rn(mul_rn(gam, pR), irR));
  const Real SL = min_num(uL - cL, uR - cR);
  const Real SR = max_num(uL + cL, uR + cR);
  // physical fluxes by the same rounded sequence on both sides
  const Real mL = mul_rn(rL, uL), mR = mul_rn(rR, uR);
  Real FL[4] = {mL, fma(mL, uL, pL), mul_rn(mL, vL), mul_rn(uL, UL[3] + pL)};
  Real FR[4] = {mR, fma(mR, uR, pR), mul_rn(mR, vR), mul_rn(uR, UR[3] + pR)};
  const Real iw = recip(SR - SL);
  const bool useL = ge0_num(SL), useR = !gt0_num(SR);
  const bool dom = solver_domain(rL, rR, pL, pR);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    // x-mirror: (L, R, S_L, S_R) -> (R', L', -S_R, -S_L) swaps the two
    // products; each is rounded on its own so the mirror face negates exactly
    const Real a = mul_rn(SR, FL[v]), b = mul_rn(SL, FR[v]);
    const Real c = mul_rn(mul_rn(SL, SR), UR[v] - UL[v]);
    Real Fm = add_rn(a - b, c) * iw;
    F[v] = useL ? FL[v] : (useR ? FR[v] : Fm);
    if (!dom) qnan(F[v]);
  }
}

// the Riemann solver of the grid (Grid::riemann: 0 HLLC, 1 HLL)
template <class Real>
__device__ __forceinline__ void riemann_x(int kind, const Real* UL, const Real* UR, Real gam,
                                          Real* F, Real& pL, Real& pR) {
  if (kind == 1) hll_x<Real>(UL, UR, gam, F, pL, pR);
  else hllc_x<Real>(UL, UR, gam, F, pL, pR);
}

// ---------------------------------------------------------------------------
// ghost cells: one kernel over all ghost cells.  The x-ghosts of interior rows
// are set from the W/E rule; the y-ghost rows (corners included) from the S/N
// rule applied to the (possibly x-ghost) cell they copy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_cell(const double* X, const Grid& g, int i, int j,
                                          double* S) {
#pragma unroll
  for (int v = 0; v < 4; ++v) S[v] = X[gidx(g, v, i, j)];
}

// the per-direction CFL rate of one cell, max((|u|+c)/dx, (|v|+c)/dy): the
// admissible step is CFL over its maximum over the cells (the minimum of
// dx/(|u|+c) and dy/(|v|+c), reduced as a maximum of rates so that each cell
// needs one reciprocal and no division).  False: no admissible step (the
// rate NaN, infinite or zero; p / rho < 0 gives NaN).
__device__ __forceinline__ bool cell_rate(const double* S, const Grid& g, double& rate) {
  const double ir = recip(S[0]);
  const double u = S[1] * ir, v = S[2] * ir;
  const double p = (g.gamma - 1.0) * (S[3] - 0.5 * (S[1] * u + S[2] * v));
  const double cs = sqrt(g.gamma * p * ir);
  const double ax = (fabs(u) + cs) * g.inv_dx, ay = (fabs(v) + cs) * g.inv_dy;
  rate = (g.dim == 1 || lt_ieee(ay, ax)) ? ax : ay;  // a NaN state makes both rates NaN
  return pos_finite(rate);
}

// the same rate on the FP32 path: from the float shadow, in float
__device__ __forceinline__ bool cell_rate(const float* S, const Grid& g, double& rate) {
  const float gam = (float)g.gamma;
  const float ir = recip(S[0]);
  const float u = S[1] * ir, v = S[2] * ir;
  const float p = (gam - 1.0f) * (S[3] - 0.5f * (S[1] * u + S[2] * v));
  const float cs = sqrt_r(gam * p * ir);
  const float ax = (fabsf(u) + cs) * (float)g.inv_dx, ay = (fabsf(v) + cs) * (float)g.inv_dy;
  const float r = (g.dim == 1 || ax > ay) ? ax : ay;
  rate = (double)r;
  return r > 0.0f && isfinite(r);
}

// the rate of cell (i, j): the double state, or its float shadow when Xf is set
__device__ __forceinline__ bool cell_rate_at(const double* X, const float* Xf, const Grid& g,
                                             int i, int j, double& rate) {
  if (Xf) {
    float S[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) S[v] = Xf[gidx(g, v, i, j)];
    return cell_rate(S, g, rate);
  }
  double S[4];
  load_cell(X, g, i, j, S);
  return cell_rate(S, g, rate);
}

// value of the x-ghost (i outside [0,nx)) of interior row j
__device__ __forceinline__ void xghost(const double* X, const Grid& g, int i, int j, double* S) {
  int side = i < 0 ? 0 : 1;
  int k = i < 0 ? -i : i - g.nx + 1;  // ghost layer 1..H
  int kind = g.bc[side];
  if (kind == 3) {
#pragma unroll
    for (int v = 0; v < 4; ++v) S[v] = g.bcU[side][v];
    return;
  }
  int src;
  if (kind == 0) src = wrapi(i, g.nx);
  else if (kind == 2) src = side == 0 ? k - 1 : g.nx - k;
  else src = side == 0 ? 0 : g.nx - 1;
  load_cell(X, g, src, j, S);
  if (kind == 2) S[1] = -S[1];
}

__device__ __forceinline__ void column_cell(const double* X, const Grid& g, int i, int j,
                                            double* S) {
  if (i < 0 || i >= g.nx) xghost(X, g, i, j, S);
  else load_cell(X, g, i, j, S);
}

// ghost cell number tid of the grid (x-ghosts of interior rows first, then
// the ghost rows, corners included), at time t; tid beyond the ghost count
// does nothing
__device__ __forceinline__ long long ghost_count(const Grid& g) {
  return (long long)g.ny * 2 * g.H + (long long)2 * g.H * (g.nx + 2 * g.H);
}

// Xf: the float shadow of X (FP32 path), filled alongside, or null
__device__ __forceinline__ void fill_ghost(double* X, float* Xf, const Grid& g, double t,
                                           long long tid) {
  const int H = g.H;
  const int nxg = g.nx + 2 * H;
  const long long nxs = (long long)g.ny * 2 * H;  // x-ghosts of interior rows
  const long long nys = (long long)2 * H * nxg;   // y-ghost rows
  if (tid >= nxs + nys) return;
  double S[4];
  int i, j;
  if (tid < nxs) {
    j = (int)(tid / (2 * H));
    int c = (int)(tid % (2 * H));
    i = c < H ? -1 - c : g.nx + (c - H);
    xghost(X, g, i, j, S);
  } else {
    long long u = tid - nxs;
    int r = (int)(u / nxg);
    i = (int)(u % nxg) - H;
    int side = r < H ? 0 : 1;  // 0: south, 1: north
    int k = r < H ? r + 1 : r - H + 1;
    j = side == 0 ? -k : g.ny - 1 + k;
    int kind = g.bc[2 + side];
    double xc = g.x0 + (i + 0.5) * g.dx;
    bool fixed = false, reflect = false;
    const double* P = nullptr;
    if (kind == 3) {
      fixed = true;
      P = g.bcU[2 + side];
    } else if (kind == 4) {
      if (xc < g.dmr_wall_x0) {
        fixed = true;
        P = g.dmr_post;
      } else {
        reflect = true;
      }
    } else if (kind == 5) {
      fixed = true;
      P = (xc < g.dmr_xs0 + g.dmr_xs_speed * t) ? g.dmr_post : g.dmr_pre;
    } else if (kind == 6) {
      // jet inflow inside the slit (cell centres), outflow elsewhere
      if (xc >= g.jet_x0 && xc <= g.jet_x1) {
        fixed = true;
        P = g.jetU[side];
      }
    } else if (kind == 2) {
      reflect = true;
    }
    if (fixed) {
#pragma unroll
      for (int v = 0; v < 4; ++v) S[v] = P[v];
    } else {
      int src;
      if (kind == 0) src = wrapi(j, g.ny);
      else if (reflect) src = side == 0 ? k - 1 : g.ny - k;
      else src = side == 0 ? 0 : g.ny - 1;
      column_cell(X, g, i, src, S);
      if (reflect) S[2] = -S[2];
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) X[gidx(g, v, i, j)] = S[v];
  if (Xf) {
#pragma unroll
    for (int v = 0; v < 4; ++v) Xf[gidx(g, v, i, j)] = (float)S[v];
  }
}

// Real copy of a ghosted state: the float shadow of the FP32 path (and of
// the FP32 adjoint), Y = (Real)X elementwise
template <class Real>
__global__ void k_to_real(const double* X, Real* Y, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    Y[t] = (Real)X[t];
}

// ---------------------------------------------------------------------------
// face-state check of cell (i, j): a state that its own stencil produced on
// one of its four faces, at the face's current radius, failed (non-finite or
// non-positive density or pressure).  Periodic seams need no care: a seam
// face's state of the cell across the seam is computed from the same data at
// the cell's own face; other ghosts' states flag nothing.
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ bool face_state_bad(const StageArgs<Real>& A, const Grid& g, int i,
                                               int j) {
  const long long wf = (long long)j * (g.nx + 1) + i;  // x face i: W face of (i, j)
  int b = (A.fbx[wf] >> 1) | A.fbx[wf + 1];            // its right / the E face's left state
  if (g.dim == 2) {
    const long long sf = (long long)j * g.nx + i;       // y face j: S face of (i, j)
    b |= (A.fby[sf] >> 1) | A.fby[sf + g.nx];
  }
  return (b & 1) != 0;
}

// ---------------------------------------------------------------------------
// the face-state tape of a recorded step (Control::stape): the states the
// step's final fluxes were solved from, so that the adjoint need not
// reconstruct them again.  Per stage: x faces (left, right states), y faces
// (lower, upper), each [4 variables][qt points][faces of that direction],
// qt the rule size of the top radius.  Null when the step records none.
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ Real* state_tape(const StageArgs<Real>& A, const Grid& g, int qt,
                                            int dir, int side) {
  Real* base = (Real*)A.sc->ctl.stape;
  if (!base) return nullptr;
  const long long nfx = (long long)(g.nx + 1) * g.ny, nfy = (long long)g.nx * (g.ny + 1);
  base += (long long)A.stage * 8 * qt * (nfx + nfy);
  return dir == 0 ? base + (long long)side * 4 * qt * nfx
                  : base + 8LL * qt * nfx + (long long)side * 4 * qt * nfy;
}

// the states UL / UR of point q of face f (of its direction) into the tape
template <class Real>
__device__ __forceinline__ void tape_states(Real* tL, Real* tR, int qt, long long nf, long long f,
                                            int q, const Real* UL, const Real* UR) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    tL[((long long)v * qt + q) * nf + f] = UL[v];
    tR[((long long)v * qt + q) * nf + f] = UR[v];
  }
}

// the same for the face between (iL, jL) and its neighbour in direction DIR
// (a periodic seam face: both copies), when the step records states
template <class Real, int DIR>
__device__ __forceinline__ void tape_face(const StageArgs<Real>& A, const Grid& g, int qt, int iL,
                                          int jL, int q, const Real* UL, const Real* UR) {
  Real* tL = state_tape<Real>(A, g, qt, DIR, 0);
  if (!tL) return;
  Real* tR = state_tape<Real>(A, g, qt, DIR, 1);
  if (DIR == 0) {
    const long long nf = (long long)(g.nx + 1) * g.ny;
    const int f = iL + 1;
    tape_states(tL, tR, qt, nf, (long long)jL * (g.nx + 1) + f, q, UL, UR);
    if (g.periodic_x && (f == 0 || f == g.nx))
      tape_states(tL, tR, qt, nf, (long long)jL * (g.nx + 1) + (f == 0 ? g.nx : 0), q, UL, UR);
  } else {
    const long long nf = (long long)g.nx * (g.ny + 1);
    const int f = jL + 1;
    tape_states(tL, tR, qt, nf, (long long)f * g.nx + iL, q, UL, UR);
    if (g.periodic_y && (f == 0 || f == g.ny))
      tape_states(tL, tR, qt, nf, (long long)(f == 0 ? g.ny : 0) * g.nx + iL, q, UL, UR);
  }
}

// ---------------------------------------------------------------------------
// first-pass faces at the top radius R.  One warp covers 32 consecutive
// cells of a row (x_faces) or a column (y_faces) and produces the 31 faces
// between them; the left/lower states come from the neighbouring lane.
// ---------------------------------------------------------------------------
// shared-memory tile of one face block: the block's cells and their
// stencils, converted to Real once, as tile[v][across][along]: "along" runs
// with the sweep (the lanes), "across" with the warps, so every stencil read
// of a warp is one contiguous row of shared memory
template <int R, class Real, int FW>
struct FaceTile {
  static constexpr int TF = kSegCells + 2 * R;
  static constexpr int TS = FW + 2 * R;
  Real t[4][TS][TF];
};

// stage the ghosted state X (any element type) around the block whose first
// cell is `first_fast` along the sweep and `first_slow` across it into the
// shared tile, as Real
template <int R, class Real, int DIR, int FW, class TX>
__device__ __forceinline__ void tile_load_at(FaceTile<R, Real, FW>& T_, const TX* X,
                                             const Grid& g, int first_fast, int first_slow) {
  constexpr int TF = FaceTile<R, Real, FW>::TF;
  constexpr int TS = FaceTile<R, Real, FW>::TS;
  constexpr int NE = TS * TF;                 // tile cells of one variable
  constexpr int NT = 32 * FW;                 // threads of the block
  constexpr int NP = (NE + NT - 1) / NT;      // tile cells per thread
  Real* tile = &T_.t[0][0][0];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int fast0 = first_fast - R;           // first tile cell along the sweep
  const int slow0 = first_slow - R;           // first tile cell across it
  // the cells this thread stages, worked out once for the four variables:
  // consecutive threads take consecutive cells along x (coalesced loads)
  long long off[NP];
  int soff[NP];
  bool ok[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int r = tid + p * NT;
    int sl, fa;
    if (DIR == 0) { sl = r / TF; fa = r - sl * TF; }
    else { fa = r / TS; sl = r - fa * TS; }
    const int i = DIR == 0 ? fast0 + fa : slow0 + sl;
    const int j = DIR == 0 ? slow0 + sl : fast0 + fa;
    ok[p] = i >= -g.H && i < g.nx + g.H && j >= -g.H && j < g.ny + g.H;
    off[p] = gidx(g, 0, i, j);  // dereferenced only when ok
    soff[p] = sl * TF + fa;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (tid + p * NT < NE)
        tile[v * NE + soff[p]] = ok[p] ? (Real)__ldg(X + off[p] + v * g.vstride) : Real(0);
}

// the tile of segment `seg` along the sweep and band `band` across it
template <int R, class Real, int DIR, int FW, class TX>
__device__ __forceinline__ void tile_load(FaceTile<R, Real, FW>& T_, const TX* X, const Grid& g,
                                          int seg, int band) {
  tile_load_at<R, Real, DIR, FW>(T_, X, g, seg * kSegFaces - 1, band * FW);
}

// states at all Gauss points of the two faces of one tile cell across the
// sweep (top radius R): SP on the +1/2 side (east / north), SM on the -1/2
// side (west / south).  (fl, sw): the cell's tile position along / across.
template <int R, class Real, int DIR, int FW>
__device__ __forceinline__ void tile_face_states(const FaceTile<R, Real, FW>& T_,
                                                 const ParityW<Real>& W, int fl, int sw,
                                                 bool live, Real (&SP)[rule_q(R)][4],
                                                 Real (&SM)[rule_q(R)][4]) {
  constexpr int N = stencil_n(R);
  constexpr int Q = rule_q(R);
  constexpr int NS = (Q + 1) / 2;
  auto& tile = T_.t;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    Real s[N];
    if (live) {
      // (a, b): offsets along x and y
      auto ld = [&](int a, int b) -> Real {
        return DIR == 0 ? tile[v][sw + b][fl + a] : tile[v][sw + a][fl + b];
      };
      parity_sums<R, Real>(ld, s);
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) s[k] = Real(0);
    }
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) {
      Real T[2][2];
      parity_dot<R, Real>(DIR == 0 ? W.cx[kk] : W.cy[kk], s, T);
      const bool middle = (Q & 1) && kk == Q / 2;
      if (DIR == 0) {
        // east / west at +g and -g
        if (middle) {
          SP[kk][v] = T[0][0] + T[1][0];
          SM[kk][v] = T[0][0] - T[1][0];
        } else {
          Real e = T[0][0] + T[0][1], o = T[1][0] + T[1][1];
          Real e2 = T[0][0] - T[0][1], o2 = T[1][0] - T[1][1];
          SP[kk][v] = e + o;            // E(+g)
          SM[kk][v] = e - o;            // W(+g)
          SP[Q - 1 - kk][v] = e2 + o2;  // E(-g)
          SM[Q - 1 - kk][v] = e2 - o2;  // W(-g)
        }
      } else {
        // north / south at +g and -g
        if (middle) {
          SP[kk][v] = T[0][0] + T[0][1];
          SM[kk][v] = T[0][0] - T[0][1];
        } else {
          Real e = T[0][0] + T[1][0], o = T[0][1] + T[1][1];
          Real e2 = T[0][0] - T[1][0], o2 = T[0][1] - T[1][1];
          SP[kk][v] = e + o;            // N(+g)
          SM[kk][v] = e - o;            // S(+g)
          SP[Q - 1 - kk][v] = e2 + o2;  // N(-g)
          SM[Q - 1 - kk][v] = e2 - o2;  // S(-g)
        }
      }
    }
  }
}

// one block of the first-pass face sweep (DIR 0: x faces, 1: y faces) over
// segment `seg` along the sweep and band `band` of FW rows/columns across it
template <int R, class Real, int DIR, int FW>
__device__ __forceinline__ void faces_block(const StageArgs<Real>& A, const Grid& g,
                                            const ParityW<Real>& W, int seg, int band,
                                            FaceTile<R, Real, FW>& T_) {
  constexpr int Q = rule_q(R);
  tile_load<R, Real, DIR, FW>(T_, A.Xr, g, seg, band);
  __syncthreads();
  const int lane = threadIdx.x, warp = threadIdx.y;
  // DIR 0: lanes along x, warp per row; DIR 1: lanes along y, warp per column
  int i, j, nlen, across;
  if (DIR == 0) {
    j = band * FW + warp;
    i = seg * kSegFaces - 1 + lane;
    nlen = g.nx;
    across = g.ny;
  } else {
    i = band * FW + warp;
    j = seg * kSegFaces - 1 + lane;
    nlen = g.ny;
    across = g.nx;
  }
  if ((DIR == 0 ? j : i) >= across) return;  // whole warp
  const int pos = DIR == 0 ? i : j;  // position along the sweep, -1 .. nlen
  const bool live = pos <= nlen;
  Real SP[Q][4], SM[Q][4];
  tile_face_states<R, Real, DIR, FW>(T_, W, lane + R, warp + R, live, SP, SM);
  // left/lower state of the face between this cell and the previous one
  Real SL[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) SL[q][v] = __shfl_up_sync(0xffffffffu, SP[q][v], 1);
  // face index = pos (between pos-1 and pos)
  if (lane == 0 || pos < 0 || pos > nlen) return;
  const Real gam = (Real)g.gamma;
  Real F[4] = {0, 0, 0, 0};
  bool badL = false, badR = false;
  auto point = [&](int q, Real* f) {
    Real pl, pr;
    if (DIR == 0) {
      riemann_x<Real>(g.riemann, SL[q], SM[q], gam, f, pl, pr);
    } else {
      Real a[4] = {SL[q][0], SL[q][2], SL[q][1], SL[q][3]};
      Real b[4] = {SM[q][0], SM[q][2], SM[q][1], SM[q][3]};
      Real h[4];
      riemann_x<Real>(g.riemann, a, b, gam, h, pl, pr);
      f[0] = h[0]; f[1] = h[2]; f[2] = h[1]; f[3] = h[3];
    }
    // face-state check: finite and positive density and pressure (the
    // solver's sound speed needs gamma p / rho > 0; NaN fails the test)
    badL |= !(pos_finite(SL[q][0]) && pos_finite(pl));
    badR |= !(pos_finite(SM[q][0]) && pos_finite(pr));
  };
  // the Gauss points in mirror pairs (g, -g), each pair summed first: a
  // mirror image of the problem that reverses the points sums alike
#pragma unroll
  for (int kk = 0; kk < (Q + 1) / 2; ++kk) {
    Real f1[4];
    point(kk, f1);
    if (Q - 1 - kk != kk) {
      Real f2[4];
      point(Q - 1 - kk, f2);
#pragma unroll
      for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], add_rn(f1[v], f2[v]), F[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], f1[v], F[v]);
    }
  }
  if (DIR == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) A.Fx[fxidx(g, v, i, j)] = F[v];
    A.fbx[(long long)j * (g.nx + 1) + i] = (uint8_t)((badL ? 1 : 0) | (badR ? 2 : 0));
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) A.Fy[fyidx(g, v, i, j)] = F[v];
    A.fby[(long long)j * g.nx + i] = (uint8_t)((badL ? 1 : 0) | (badR ? 2 : 0));
  }
  // a recorded step keeps the states for its adjoint
  if (Real* tL = state_tape<Real>(A, g, Q, DIR, 0)) {
    Real* tR = state_tape<Real>(A, g, Q, DIR, 1);
    const long long nf = DIR == 0 ? (long long)(g.nx + 1) * g.ny : (long long)g.nx * (g.ny + 1);
    const long long f = DIR == 0 ? (long long)j * (g.nx + 1) + i : (long long)j * g.nx + i;
#pragma unroll
    for (int q = 0; q < Q; ++q) tape_states(tL, tR, Q, nf, f, q, SL[q], SM[q]);
  }
}

template <int R, class Real, int DIR, int FW>
__global__ void __launch_bounds__(32 * FW) k_faces(StageArgs<Real> A, Grid g,
                                                   const __grid_constant__ ParityW<Real> W) {
  pdl_wait();
  pdl_trigger();
  __shared__ FaceTile<R, Real, FW> tile;
  faces_block<R, Real, DIR, FW>(A, g, W, DIR == 0 ? blockIdx.x : blockIdx.y,
                                DIR == 0 ? blockIdx.y : blockIdx.x, tile);
}

// ---------------------------------------------------------------------------
// both first-pass face sweeps in one block (two-dimensional grids).  A block
// of 8 warps covers 8 rows of a 32-cell segment: lane l, warp w hold cell
// (i0 + l, j0 + w), i0 = 31 seg - 1, j0 = 7 band - 1, so segments overlap by
// one column and bands by one row.  Each cell forms its parity sums once per
// variable and from them both its x states (E/W, kept in registers for the
// x faces, taken from the neighbouring lane by shuffle) and its y states
// (N/S, written to shared memory for the y faces between consecutive rows).
// A thread with l, w >= 1 then solves the x face between (i-1, j) and
// (i, j) and the y face between (i, j-1) and (i, j).  The arithmetic of
// every state and flux is that of the separate sweeps (k_faces), so the
// fluxes are the same bit for bit; y fluxes are stored with lanes along x.
// ---------------------------------------------------------------------------
constexpr int kXYRows = 8;               // cell rows of a fused face block (its warps)
constexpr int kXYBand = kXYRows - 1;     // face rows a block owns

template <int R, class Real>
struct XYShared {
  FaceTile<R, Real, kXYRows> tile;
  Real ys[2][rule_q(R)][4][kXYRows][32];  // [N, S][point][variable][row][lane]
};

// one fused block: segment `seg` (31 x faces) and band `band` (7 rows of
// faces) of the grid
template <int R, class Real>
__device__ __forceinline__ void faces_xy_block(const StageArgs<Real>& A, const Grid& g,
                                               const ParityW<Real>& W, int seg, int band,
                                               XYShared<R, Real>& S) {
  constexpr int N = stencil_n(R);
  constexpr int Q = rule_q(R);
  constexpr int NS = (Q + 1) / 2;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int i0 = seg * kSegFaces - 1, j0 = band * kXYBand - 1;
  tile_load_at<R, Real, 0, kXYRows>(S.tile, A.Xr, g, i0, j0);
  __syncthreads();
  const int i = i0 + lane, j = j0 + warp;
  // rows beyond the last y face take no part (their states feed nothing)
  const bool row_live = j <= g.ny;
  const bool xrow = warp >= 1 && j < g.ny;  // this warp's x faces are the block's
  Real SP[Q][4], SM[Q][4];
  auto& tile = S.tile.t;
  const int fl = lane + R, sw = warp + R;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    Real s[N];
    if (row_live) {
      auto ld = [&](int a, int b) -> Real { return tile[v][sw + b][fl + a]; };
      parity_sums<R, Real>(ld, s);
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) s[k] = Real(0);
    }
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) {
      const bool middle = (Q & 1) && kk == Q / 2;
      if (xrow) {
        // east / west at +g and -g (the x sweep's butterflies)
        Real T[2][2];
        parity_dot<R, Real>(W.cx[kk], s, T);
        if (middle) {
          SP[kk][v] = T[0][0] + T[1][0];
          SM[kk][v] = T[0][0] - T[1][0];
        } else {
          Real e = T[0][0] + T[0][1], o = T[1][0] + T[1][1];
          Real e2 = T[0][0] - T[0][1], o2 = T[1][0] - T[1][1];
          SP[kk][v] = e + o;
          SM[kk][v] = e - o;
          SP[Q - 1 - kk][v] = e2 + o2;
          SM[Q - 1 - kk][v] = e2 - o2;
        }
      }
      // north / south at +g and -g (the y sweep's butterflies), to shared memory
      Real T[2][2];
      parity_dot<R, Real>(W.cy[kk], s, T);
      if (middle) {
        S.ys[0][kk][v][warp][lane] = T[0][0] + T[0][1];
        S.ys[1][kk][v][warp][lane] = T[0][0] - T[0][1];
      } else {
        Real e = T[0][0] + T[1][0], o = T[0][1] + T[1][1];
        Real e2 = T[0][0] - T[1][0], o2 = T[0][1] - T[1][1];
        S.ys[0][kk][v][warp][lane] = e + o;
        S.ys[1][kk][v][warp][lane] = e - o;
        S.ys[0][Q - 1 - kk][v][warp][lane] = e2 + o2;
        S.ys[1][Q - 1 - kk][v][warp][lane] = e2 - o2;
      }
    }
  }
  const Real gam = (Real)g.gamma;
  // x faces: the left state from the neighbouring lane
  if (xrow) {
    Real SL[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) SL[q][v] = __shfl_up_sync(0xffffffffu, SP[q][v], 1);
    if (lane >= 1 && i <= g.nx) {
      Real F[4] = {0, 0, 0, 0};
      bool badL = false, badR = false;
      auto point = [&](int q, Real* f) {
        Real pl, pr;
        riemann_x<Real>(g.riemann, SL[q], SM[q], gam, f, pl, pr);
        badL |= !(pos_finite(SL[q][0]) && pos_finite(pl));
        badR |= !(pos_finite(SM[q][0]) && pos_finite(pr));
      };
#pragma unroll
      for (int kk = 0; kk < NS; ++kk) {
        Real f1[4];
        point(kk, f1);
        if (Q - 1 - kk != kk) {
          Real f2[4];
          point(Q - 1 - kk, f2);
#pragma unroll
          for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], add_rn(f1[v], f2[v]), F[v]);
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], f1[v], F[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) A.Fx[fxidx(g, v, i, j)] = F[v];
      A.fbx[(long long)j * (g.nx + 1) + i] = (uint8_t)((badL ? 1 : 0) | (badR ? 2 : 0));
      if (Real* tL = state_tape<Real>(A, g, Q, 0, 0)) {
        Real* tR = state_tape<Real>(A, g, Q, 0, 1);
        const long long nf = (long long)(g.nx + 1) * g.ny, f = (long long)j * (g.nx + 1) + i;
#pragma unroll
        for (int q = 0; q < Q; ++q) tape_states(tL, tR, Q, nf, f, q, SL[q], SM[q]);
      }
    }
  }
  __syncthreads();
  // y faces: the lower state from the row below, both from shared memory
  if (warp >= 1 && lane >= 1 && i < g.nx && j <= g.ny) {
    Real F[4] = {0, 0, 0, 0};
    bool badL = false, badR = false;
    auto point = [&](int q, Real* f) {
      Real a[4], b[4];
      a[0] = S.ys[0][q][0][warp - 1][lane];
      a[1] = S.ys[0][q][2][warp - 1][lane];
      a[2] = S.ys[0][q][1][warp - 1][lane];
      a[3] = S.ys[0][q][3][warp - 1][lane];
      b[0] = S.ys[1][q][0][warp][lane];
      b[1] = S.ys[1][q][2][warp][lane];
      b[2] = S.ys[1][q][1][warp][lane];
      b[3] = S.ys[1][q][3][warp][lane];
      Real h[4], pl, pr;
      riemann_x<Real>(g.riemann, a, b, gam, h, pl, pr);
      f[0] = h[0]; f[1] = h[2]; f[2] = h[1]; f[3] = h[3];
      badL |= !(pos_finite(a[0]) && pos_finite(pl));
      badR |= !(pos_finite(b[0]) && pos_finite(pr));
    };
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) {
      Real f1[4];
      point(kk, f1);
      if (Q - 1 - kk != kk) {
        Real f2[4];
        point(Q - 1 - kk, f2);
#pragma unroll
        for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], add_rn(f1[v], f2[v]), F[v]);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) F[v] = fma(W.w[kk], f1[v], F[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) A.Fy[fyidx(g, v, i, j)] = F[v];
    A.fby[(long long)j * g.nx + i] = (uint8_t)((badL ? 1 : 0) | (badR ? 2 : 0));
    if (Real* tL = state_tape<Real>(A, g, Q, 1, 0)) {
      Real* tR = state_tape<Real>(A, g, Q, 1, 1);
      const long long nf = (long long)g.nx * (g.ny + 1), f = (long long)j * g.nx + i;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        Real UL[4], UR[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          UL[v] = S.ys[0][q][v][warp - 1][lane];
          UR[v] = S.ys[1][q][v][warp][lane];
        }
        tape_states(tL, tR, Q, nf, f, q, UL, UR);
      }
    }
  }
}

// resident blocks of the fused face kernel: FP64 2 (128 registers), FP32 4
template <class Real>
constexpr int xy_min_blocks() { return sizeof(Real) == sizeof(double) ? 2 : 4; }

template <int R, class Real>
__global__ void __launch_bounds__(32 * kXYRows, xy_min_blocks<Real>()) k_faces_xy(StageArgs<Real> A, Grid g,
                                                           const __grid_constant__ ParityW<Real> W) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char xy_smem[];
  XYShared<R, Real>& S = *reinterpret_cast<XYShared<R, Real>*>(xy_smem);
  faces_xy_block<R, Real>(A, g, W, blockIdx.x, blockIdx.y, S);
}

// ---------------------------------------------------------------------------
// detection, Steps 4-9 (eqs. CAD, PAD, divV, gradP, plateau, DMP_RK,
// u2_curvature, u2_a, u2_b) on the candidate Y of cell (i,j) with the ghosted
// stage input X.  Returns true for a troubled cell.
// ---------------------------------------------------------------------------
// a detection constant in the precision of the tests (Detect holds both)
template <class Real>
__device__ __forceinline__ Real det_c(double d, float f);
template <>
__device__ __forceinline__ double det_c<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float det_c<float>(double, float f) { return f; }

// a double in the precision of the tests: FP32 rounds it on the integer pipes
template <class Real>
__device__ __forceinline__ Real to_real(double x);
template <>
__device__ __forceinline__ double to_real<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_real<float>(double x) { return fpb_double_to_float_rn(x); }

template <class Real>
__device__ __forceinline__ Real xload(const Real* X, const Grid& g, int v, int i, int j) {
  return __ldg(X + gidx(g, v, i, j));
}

// X(v, a, b): variable v of the ghosted stage input at (i + a, j + b), in
// Real; every call below has constant offsets once the loops are unrolled
template <class Real, class LX>
__device__ __forceinline__ bool troubled_at(const LX& X, const Grid& g, const Detect& D,
                                            const Real* d2x, const Real* d2y, const double* Yd) {
  const Real gm1 = det_c<Real>(D.gm1, D.gm1_f);
  Real Y[4] = {to_real<Real>(Yd[0]), to_real<Real>(Yd[1]), to_real<Real>(Yd[2]),
               to_real<Real>(Yd[3])};
  Real rho = Y[0];
  Real p = gm1 * (Y[3] - Real(0.5) * (Y[1] * Y[1] + Y[2] * Y[2]) * recip(Y[0]));
  if (!finite_r(rho) || !finite_r(p)) return true;    // Step 4, CAD
  if (!gt0_num(rho) || !gt0_num(p)) return true;       // Step 5, PAD
  const bool two = g.dim == 2;  // 1D: the x terms and the W/E neighbours only
  if (D.csd_on) {                                      // Step 6, CSD
    Real rE = X(0, 1, 0), rW = X(0, -1, 0);
    Real rN = X(0, 0, 1), rS = X(0, 0, -1);
    Real mxE = X(1, 1, 0), mxW = X(1, -1, 0);
    Real myE = X(2, 1, 0), myW = X(2, -1, 0);
    Real mxN = X(1, 0, 1), mxS = X(1, 0, -1);
    Real myN = X(2, 0, 1), myS = X(2, 0, -1);
    Real eE = X(3, 1, 0), eW = X(3, -1, 0);
    Real eN = X(3, 0, 1), eS = X(3, 0, -1);
    Real iE = recip(rE), iW = recip(rW), iN = recip(rN), iS = recip(rS);
    // one rounded sequence for every neighbour: mirror neighbours agree bitwise
    const Real SE[4] = {rE, mxE, myE, eE}, SW[4] = {rW, mxW, myW, eW};
    const Real SN[4] = {rN, mxN, myN, eN}, SS[4] = {rS, mxS, myS, eS};
    Real uE, uW, vN, vS, tmp;
    Real pE = pressure_ir(SE, iE, gm1, uE, tmp);
    Real pW = pressure_ir(SW, iW, gm1, uW, tmp);
    Real pN = pressure_ir(SN, iN, gm1, tmp, vN);
    Real pS = pressure_ir(SS, iS, gm1, tmp, vS);
    const Real hx = det_c<Real>(D.hx, D.hx_f), hy = det_c<Real>(D.hy, D.hy_f);
    Real mx_ = lt_ieee(pE, pW) ? pE : pW, my_ = lt_ieee(pN, pS) ? pN : pS;
    Real divV = (uE - uW) * hx, gradP = fabs(pE - pW) * hx * recip(mx_);
    if (two) {
      divV += (vN - vS) * hy;
      gradP += fabs(pN - pS) * hy * recip(my_);
    }
    if (le_ieee(-det_c<Real>(D.sigma_v, D.sigma_v_f), divV) &&
        le_ieee(gradP, det_c<Real>(D.sigma_p, D.sigma_p_f)))
      return false;
  }
  Real r0 = X(0, 0, 0);
  Real rmin = r0, rmax = r0;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, 1, -1};
  const int nnb = two ? 4 : 2;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (m >= nnb) break;
    Real r = X(0, di[m], dj[m]);
    rmin = lt_ieee(r, rmin) ? r : rmin;
    rmax = lt_ieee(rmax, r) ? r : rmax;
  }
  if (lt_ieee(rmax - rmin, det_c<Real>(D.plateau_thr, D.plateau_thr_f))) return false;  // Step 7
  if (le_ieee(rmin, rho) && le_ieee(rho, rmax)) return false;     // Step 8, DMP
  // Step 9, u2 with the App. B second-derivative weights (R=1 stencil in
  // the order b=-1: (0,-1); b=0: (-1,0),(0,0),(1,0); b=1: (0,1))
  const int ci[5] = {0, -1, 1, 0, 0}, cj[5] = {0, 0, 0, 1, -1};
  const Real delta = det_c<Real>(D.delta, D.delta_f);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    if (d == 1 && !two) break;
    const Real* w = d == 0 ? d2x : d2y;
    Real cmin = Real(0), cmax = Real(0);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      if (m >= 1 + nnb) break;
      const int a = ci[m], b = cj[m];
      // mirror pairs (S, N) and (W, E) summed first, each product rounded on
      // its own: a mirror-symmetric state gives the same curvature bit for bit
      const Real ks = add_rn(mul_rn(w[0], X(0, a, b - 1)), mul_rn(w[4], X(0, a, b + 1)));
      const Real kw = add_rn(mul_rn(w[1], X(0, a - 1, b)), mul_rn(w[3], X(0, a + 1, b)));
      Real k = add_rn(add_rn(ks, kw), mul_rn(w[2], X(0, a, b)));
      if (m == 0) {
        cmin = k;
        cmax = k;
      } else {
        cmin = lt_ieee(k, cmin) ? k : cmin;
        cmax = lt_ieee(cmax, k) ? k : cmax;
      }
    }
    bool same = lt_ieee(-delta, cmin * cmax);
    Real acmax = fabs(cmax), acmin = fabs(cmin);
    bool ua = same && lt_ieee(lt_ieee(acmin, acmax) ? acmax : acmin, delta);
    // |Cmin|/|Cmax| >= 1/2 written without the division; equal for every
    // non-NaN input once (a) is taken into account
    bool ub = same && le_ieee(Real(0.5) * acmax, acmin);
    if (!(ua || ub)) return true;
  }
  return false;
}

// X: the ghosted stage input in Real; the loads are issued as the tests
// reach them (the first pass: many cells in flight hide their latency)
template <class Real>
__device__ bool troubled(const Real* X, const Grid& g, const Detect& D, const Real* d2x,
                         const Real* d2y, int i, int j, const double* Yd) {
  auto lx = [&](int v, int a, int b) -> Real { return xload<Real>(X, g, v, i + a, j + b); };
  return troubled_at<Real>(lx, g, D, d2x, d2y, Yd);
}

// slot of offset (a, b) in the diamond |a| + |b| <= 2 (13 cells)
__host__ __device__ constexpr int diamond2_slot(int a, int b) {
  return b == -2 ? 0 : b == -1 ? 2 + a : b == 0 ? 6 + a : b == 1 ? 10 + a : 12;
}

// the same tests with every value they may read loaded first, in one batch:
// the densities of the diamond |a| + |b| <= 2 and the momenta and energies
// of the four face neighbours.  For the MOOD loop, whose few cells per
// iteration leave the latency of dependent loads exposed.
template <class Real>
__device__ bool troubled_prefetched(const Real* X, const Grid& g, const Detect& D,
                                    const Real* d2x, const Real* d2y, int i, int j,
                                    const double* Yd) {
  Real r[13], m[3][4];
#pragma unroll
  for (int b = -2; b <= 2; ++b) {
    const int hb = 2 - (b < 0 ? -b : b);
#pragma unroll
    for (int a = -hb; a <= hb; ++a) r[diamond2_slot(a, b)] = xload<Real>(X, g, 0, i + a, j + b);
  }
  const int fa[4] = {1, -1, 0, 0}, fb[4] = {0, 0, 1, -1};
#pragma unroll
  for (int v = 1; v < 4; ++v)
#pragma unroll
    for (int k = 0; k < 4; ++k) m[v - 1][k] = xload<Real>(X, g, v, i + fa[k], j + fb[k]);
  auto lx = [&](int v, int a, int b) -> Real {
    if (v == 0) return r[diamond2_slot(a, b)];
    const int k = a == 1 ? 0 : a == -1 ? 1 : b == 1 ? 2 : 3;
    return m[v - 1][k];
  };
  return troubled_at<Real>(lx, g, D, d2x, d2y, Yd);
}

// candidate of eq. fvm_discrete and the SSP-RK3 combination (eq. rk3) of cell (i,j)
// the stage's flux-difference coefficients h dt / dx and h dt / dy
struct StageC {
  double cx, cy;
};
template <class Real>
__device__ __forceinline__ StageC stage_coeffs(const StageArgs<Real>& A, const Grid& g,
                                               double dt) {
  const double hdt = A.h * dt;
  return StageC{hdt * g.inv_dx, hdt * g.inv_dy};
}

// per variable two differences and two fmas
template <class Real>
__device__ __forceinline__ void candidate(const StageArgs<Real>& A, const Grid& g, int i, int j,
                                          StageC k, double* Y) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double fe = A.Fx[fxidx(g, v, i + 1, j)], fw = A.Fx[fxidx(g, v, i, j)];
    double gn = A.Fy[fyidx(g, v, i, j + 1)], gs = A.Fy[fyidx(g, v, i, j)];
    Y[v] = fma(-k.cx, fe - fw, fma(-k.cy, gn - gs, A.X[gidx(g, v, i, j)]));
  }
}
template <class Real>
__device__ __forceinline__ void candidate(const StageArgs<Real>& A, const Grid& g, int i, int j,
                                          double dt, double* Y) {
  candidate<Real>(A, g, i, j, stage_coeffs<Real>(A, g, dt), Y);
}

template <class Real>
__device__ __forceinline__ void combine_store(const StageArgs<Real>& A, const Grid& g, int i,
                                              int j, const double* Y) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    long long k = gidx(g, v, i, j);
    // the first stage's combination is the candidate itself (ca = 0, cb = 1)
    const double o = A.ca != 0.0 ? fma(A.ca, A.U0[k], A.cb * Y[v])
                                 : (A.cb == 1.0 ? Y[v] : A.cb * Y[v]);
    A.out[k] = o;
    if constexpr (sizeof(Real) == sizeof(float)) A.outr[k] = fpb_double_to_float_rn(o);
    if (A.out2) A.out2[k] = fma(A.wa, A.W[k], A.wb * Y[v]);
  }
}

// append to a queue with one atomic per warp
__device__ __forceinline__ void queue_push(bool flag, int cell, int* queue, int* count) {
  unsigned act = __activemask();
  unsigned m = __ballot_sync(act, flag);
  if (m == 0) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(act, base, leader);
  if (flag) queue[base + __popc(m & ((1u << lane) - 1u))] = cell;
}

// first-pass update of cell (i,j) (if in range): candidate, detection,
// RK combination; troubled cells go to the queue as cell_off + local index.
// D and d2x/d2y are the detection constants and App. B weights of the grid.
template <class Real>
__device__ __forceinline__ void update_cell_w(const StageArgs<Real>& A, const Grid& g,
                                              const Detect& D, const DirectW<Real>& Wd,
                                              const Real* d2x, const Real* d2y, int i, int j,
                                              int cell_off, StageC k) {
  const bool in = i < g.nx && j < g.ny;
  bool bad = false;
  int c = 0;
  if (in) {
    c = cidx(g, i, j);
    double Y[4];
    candidate<Real>(A, g, i, j, k, Y);
    const int top = Wd.top;
    if (top != 0) {
      bad = face_state_bad<Real>(A, g, i, j) || troubled<Real>(A.Xr, g, D, d2x, d2y, i, j, Y);
    } else {
      Real y[4] = {(Real)Y[0], (Real)Y[1], (Real)Y[2], (Real)Y[3]};
      Real p = (Real)(g.gamma - 1.0) * (y[3] - Real(0.5) * (y[1] * y[1] + y[2] * y[2]) / y[0]);
      if (!(y[0] > Real(0)) || !(p > Real(0))) atomicAdd(&A.scw->nfog_pad[A.stage], 1);
    }
    A.ord[c] = (uint8_t)top;
    A.first[c] = (uint8_t)bad;
    combine_store<Real>(A, g, i, j, Y);
  }
  queue_push(bad, cell_off + c, A.queue, A.qcount);
}

template <class Real>
__global__ void __launch_bounds__(256) k_update_first(StageArgs<Real> A, Grid g, Detect D,
                                                      const __grid_constant__ DirectW<Real> Wd) {
  pdl_wait();
  pdl_trigger();
  // the stage coefficients once per block: FP64 work is charged per warp
  // instruction, so a value every warp computed would cost every warp
  __shared__ StageC k;
  if (threadIdx.x == 0 && threadIdx.y == 0) k = stage_coeffs<Real>(A, g, A.sc->dt);
  __syncthreads();
  update_cell_w<Real>(A, g, D, Wd, Wd.d2x, Wd.d2y, blockIdx.x * blockDim.x + threadIdx.x,
                      blockIdx.y * blockDim.y + threadIdx.y, 0, k);
}

// ---------------------------------------------------------------------------
// MOOD iteration kernels
// ---------------------------------------------------------------------------
// neighbour of (i,j) in direction d (0 W, 1 E, 2 S, 3 N) with periodic wrap;
// returns -1 beyond a non-periodic boundary
__device__ __forceinline__ int neighbour(const Grid& g, int i, int j, int d) {
  int a = i + (d == 0 ? -1 : d == 1 ? 1 : 0);
  int b = j + (d == 2 ? -1 : d == 3 ? 1 : 0);
  if (a < 0 || a >= g.nx) {
    if (!g.periodic_x) return -1;
    a = wrapi(a, g.nx);
  }
  if (b < 0 || b >= g.ny) {
    if (!g.periodic_y) return -1;
    b = wrapi(b, g.ny);
  }
  return cidx(g, a, b);
}

// radius of a possibly-ghost cell now and before this iteration's lowering
__device__ __forceinline__ void radius_pair(const Grid& g, const uint8_t* ord, const uint32_t* stamp,
                                            uint32_t cur, const Cascade& C, int i, int j,
                                            int& now, int& before) {
  const int top = C.top;
  if (i < 0 || i >= g.nx) {
    if (!g.periodic_x) { now = before = top; return; }
    i = wrapi(i, g.nx);
  }
  if (j < 0 || j >= g.ny) {
    if (!g.periodic_y) { now = before = top; return; }
    j = wrapi(j, g.ny);
  }
  int c = cidx(g, i, j);
  now = ord[c];
  before = stamp[c] == cur ? C.prev[now] : now;
}

// direct reconstruction of one face state at radius K (eq. gp_reconstructor)
// T: storage type of the ghosted state (Real, or double read into Real)
template <int K, class Real, class T = Real>
__device__ __forceinline__ void recon_direct(const T* X, const Grid& g, const Real* z, int i,
                                             int j, Real* S) {
  // row by row, each row from its centre out in x-mirror pairs (a, -a) with
  // every product rounded on its own: the x-mirror image of the problem,
  // whose weights are the mirrored ones, gives the mirrored state bit for bit
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T* Xv = X + (long long)v * g.vstride + (long long)(j + g.H) * g.pitch + (i + g.H);
    Real s = Real(0);
    int row = 0;  // stencil index of the row's first cell
#pragma unroll
    for (int b = -K; b <= K; ++b) {
      const int hb = K - (b < 0 ? -b : b);
      const int mid = row + hb;  // (0, b)
      const T* Xr = Xv + (long long)b * g.pitch;
      Real t = mul_rn(z[mid], (Real)__ldg(Xr));
#pragma unroll
      for (int a = 1; a <= hb; ++a)
        t = add_rn(t, add_rn(mul_rn(z[mid + a], (Real)__ldg(Xr + a)),
                             mul_rn(z[mid - a], (Real)__ldg(Xr - a))));
      s = add_rn(s, t);
      row += 2 * hb + 1;
    }
    S[v] = s;
  }
}

// Riemann flux at Gauss point q of the face between cell (iL,jL) and its
// neighbour (iR,jR) in direction DIR at radius K; badL / badR gather the
// face-state check of the two reconstructed states
template <int K, class Real, int DIR>
__device__ __forceinline__ void face_point(const Real* X, const Grid& g, const DirectW<Real>& Wd,
                                           int iL, int jL, int q, Real* f, bool& badL,
                                           bool& badR, Real* sUL = nullptr,
                                           Real* sUR = nullptr) {
  const int iR = iL + (DIR == 0), jR = jL + (DIR == 1);
  const Real gam = (Real)g.gamma;
  Real UL[4], UR[4];
  if (K == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      UL[v] = __ldg(X + gidx(g, v, iL, jL));
      UR[v] = __ldg(X + gidx(g, v, iR, jR));
    }
  } else {
    // faces: 0 E, 1 W, 2 N, 3 S
    recon_direct<K, Real>(X, g, Wd.z[K][DIR == 0 ? 0 : 2][q], iL, jL, UL);
    recon_direct<K, Real>(X, g, Wd.z[K][DIR == 0 ? 1 : 3][q], iR, jR, UR);
  }
  Real pl, pr;
  if (DIR == 0) {
    riemann_x<Real>(g.riemann, UL, UR, gam, f, pl, pr);
  } else {
    Real a[4] = {UL[0], UL[2], UL[1], UL[3]};
    Real b[4] = {UR[0], UR[2], UR[1], UR[3]};
    Real h[4];
    riemann_x<Real>(g.riemann, a, b, gam, h, pl, pr);
    f[0] = h[0]; f[1] = h[2]; f[2] = h[1]; f[3] = h[3];
  }
  badL |= !(pos_finite(UL[0]) && pos_finite(pl));
  badR |= !(pos_finite(UR[0]) && pos_finite(pr));
  if (sUL) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sUL[v] = UL[v];
      sUR[v] = UR[v];
    }
  }
}

// face between cell (iL,jL) and its neighbour (iR,jR) in direction DIR at radius K
template <int K, class Real, int DIR>
__device__ void face_at(const Real* X, const Grid& g, const DirectW<Real>& Wd, int iL, int jL,
                        Real* F, bool& badL, bool& badR) {
  constexpr int Q = rule_q(K);
  F[0] = F[1] = F[2] = F[3] = Real(0);
  badL = badR = false;
  // mirror pairs (g, -g) summed first, in the order of the first-pass sweep
#pragma unroll
  for (int kk = 0; kk < (Q + 1) / 2; ++kk) {
    Real f1[4];
    face_point<K, Real, DIR>(X, g, Wd, iL, jL, kk, f1, badL, badR);
    if (Q - 1 - kk != kk) {
      Real f2[4];
      face_point<K, Real, DIR>(X, g, Wd, iL, jL, Q - 1 - kk, f2, badL, badR);
#pragma unroll
      for (int v = 0; v < 4; ++v) F[v] = fma(Wd.w[K][kk], add_rn(f1[v], f2[v]), F[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) F[v] = fma(Wd.w[K][kk], f1[v], F[v]);
    }
  }
}

// the flux and state-check bits of the face between (iL,jL) and its
// neighbour in direction DIR; a periodic seam face writes both copies
template <class Real, int DIR>
__device__ __forceinline__ void store_face(const StageArgs<Real>& A, const Grid& g, int iL,
                                           int jL, const Real* F, uint8_t bits) {
  const int iR = iL + (DIR == 0), jR = jL + (DIR == 1);
  if (DIR == 0) {
    int f = iR;  // face index
#pragma unroll
    for (int v = 0; v < 4; ++v) A.Fx[fxidx(g, v, f, jL)] = F[v];
    A.fbx[(long long)jL * (g.nx + 1) + f] = bits;
    if (g.periodic_x && (f == 0 || f == g.nx)) {
      int f2 = f == 0 ? g.nx : 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) A.Fx[fxidx(g, v, f2, jL)] = F[v];
      A.fbx[(long long)jL * (g.nx + 1) + f2] = bits;
    }
  } else {
    int f = jR;
#pragma unroll
    for (int v = 0; v < 4; ++v) A.Fy[fyidx(g, v, iL, f)] = F[v];
    A.fby[(long long)f * g.nx + iL] = bits;
    if (g.periodic_y && (f == 0 || f == g.ny)) {
      int f2 = f == 0 ? g.ny : 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) A.Fy[fyidx(g, v, iL, f2)] = F[v];
      A.fby[(long long)f2 * g.nx + iL] = bits;
    }
  }
}

// face f (0 W, 1 E, 2 S, 3 N) of queued cell c: recompute it if its EDP1
// radius changed; the face shared with another queued cell is done by the
// west/south one
// false when the face needs no work; else its left/lower cell (iL, jL) and
// its new EDP1 radius K
template <class Real>
__device__ __forceinline__ bool mood_face_plan(const StageArgs<Real>& A, const Grid& g,
                                               const Cascade& C, const uint32_t* stamp,
                                               uint32_t cur, int c, int f, int& iL, int& jL,
                                               int& K) {
  const int i = c % g.nx, j = c / g.nx;
  if (f >= 2 && g.dim == 1) return false;  // no y faces in 1D
  // every load of the decision depends on c alone: all are issued before
  // the first test, so that one memory latency covers them
  bool other = false;  // the face is the other queued cell's
  if (f == 0 || f == 2) {
    int nb = neighbour(g, i, j, f);
    other = nb >= 0 && stamp[nb] == cur;
  }
  iL = i;
  jL = j;
  if (f == 0) iL = i - 1;
  if (f == 2) jL = j - 1;
  const int iR = iL + (f < 2), jR = jL + (f >= 2);
  int nl, bl, nr, br;
  radius_pair(g, A.ord, stamp, cur, C, iL, jL, nl, bl);
  radius_pair(g, A.ord, stamp, cur, C, iR, jR, nr, br);
  if (other) return false;
  K = nl < nr ? nl : nr;
  const int Kold = bl < br ? bl : br;
  return K != Kold;  // else the EDP1 order of this face is unchanged
}

// one Gauss point of a face recomputed by the MOOD loop, with the radius K
// and the direction (0 x, 1 y) as run-time values: the lanes of one warp
// hold faces of both directions and of several radii, and a compiled
// variant per (K, direction) would run each variant present in the warp one
// after the other, Riemann solver included.  One path for all: the stencil
// rows beyond K are predicated off, and the y direction swaps the momenta
// around the x solver by selects.  The arithmetic is that of
// face_point<K, Real, DIR> (recon_direct's order, the same solver), so the
// flux is the same bit for bit.  z: this point's weights of the left and
// right states ([K][face][q][.] of DirectW, staged in shared memory).
template <class Real>
__device__ __forceinline__ void recon_rt(const Real* X, const Grid& g, const Real* zL,
                                         const Real* zR, int K, int iL, int jL, int iR, int jR,
                                         Real* UL, Real* UR) {
  // the stencil rows and their mirror pairs as loops that run K deep, the
  // eight (side, variable) sums of one term side by side; each sum sees the
  // operations of recon_direct<K> in their order
  const long long vs = g.vstride;
  const Real* XL = X + (long long)(jL + g.H) * g.pitch + (iL + g.H);
  const Real* XR = X + (long long)(jR + g.H) * g.pitch + (iR + g.H);
  Real sL[4], sR[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) sL[v] = sR[v] = Real(0);
  int row = 0;  // stencil index of the row's first cell
#pragma unroll 1
  for (int b = -K; b <= K; ++b) {
    const int hb = K - (b < 0 ? -b : b);
    const int mid = row + hb;  // (0, b)
    const Real* L0 = XL + (long long)b * g.pitch;
    const Real* R0 = XR + (long long)b * g.pitch;
    Real tL[4], tR[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      tL[v] = mul_rn(zL[mid], __ldg(L0 + v * vs));
      tR[v] = mul_rn(zR[mid], __ldg(R0 + v * vs));
    }
#pragma unroll 1
    for (int a = 1; a <= hb; ++a) {
      const Real lp = zL[mid + a], lm = zL[mid - a], rp = zR[mid + a], rm = zR[mid - a];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        tL[v] = add_rn(tL[v], add_rn(mul_rn(lp, __ldg(L0 + v * vs + a)),
                                     mul_rn(lm, __ldg(L0 + v * vs - a))));
        tR[v] = add_rn(tR[v], add_rn(mul_rn(rp, __ldg(R0 + v * vs + a)),
                                     mul_rn(rm, __ldg(R0 + v * vs - a))));
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sL[v] = add_rn(sL[v], tL[v]);
      sR[v] = add_rn(sR[v], tR[v]);
    }
    row += 2 * hb + 1;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    UL[v] = K == 0 ? __ldg(XL + v * vs) : sL[v];
    UR[v] = K == 0 ? __ldg(XR + v * vs) : sR[v];
  }
}

template <class Real>
__device__ __forceinline__ void face_point_rt(int K, int dir, const Real* X, const Grid& g,
                                              const Real* zL, const Real* zR, int iL, int jL,
                                              Real* f, bool& badL, bool& badR, Real* sUL,
                                              Real* sUR) {
  const int iR = iL + (dir == 0), jR = jL + (dir == 1);
  Real UL[4], UR[4];
  recon_rt<Real>(X, g, zL, zR, K, iL, jL, iR, jR, UL, UR);
  const bool y = dir != 0;
  const Real a[4] = {UL[0], y ? UL[2] : UL[1], y ? UL[1] : UL[2], UL[3]};
  const Real b[4] = {UR[0], y ? UR[2] : UR[1], y ? UR[1] : UR[2], UR[3]};
  Real h[4], pl, pr;
  riemann_x<Real>(g.riemann, a, b, (Real)g.gamma, h, pl, pr);
  f[0] = h[0];
  f[1] = y ? h[2] : h[1];
  f[2] = y ? h[1] : h[2];
  f[3] = h[3];
  badL |= !(pos_finite(UL[0]) && pos_finite(pl));
  badR |= !(pos_finite(UR[0]) && pos_finite(pr));
  if (sUL) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sUL[v] = UL[v];
      sUR[v] = UR[v];
    }
  }
}

// the compiled variant of radius K (the FP32 path: its arithmetic is cheap
// next to the run-time loops' overhead)
template <class Real, int DIR>
__device__ __forceinline__ void face_point_k(int K, const Real* X, const Grid& g,
                                             const DirectW<Real>& Wd, int iL, int jL, int q,
                                             Real* f, bool& bl, bool& br, Real* sUL,
                                             Real* sUR) {
  switch (K) {
    case 0: face_point<0, Real, DIR>(X, g, Wd, iL, jL, q, f, bl, br, sUL, sUR); break;
    case 1: face_point<1, Real, DIR>(X, g, Wd, iL, jL, q, f, bl, br, sUL, sUR); break;
    case 2: face_point<2, Real, DIR>(X, g, Wd, iL, jL, q, f, bl, br, sUL, sUR); break;
    default: face_point<3, Real, DIR>(X, g, Wd, iL, jL, q, f, bl, br, sUL, sUR); break;
  }
}

// DirectW's reconstruction weights, staged in shared memory by the FP64
// MOOD kernel: the lanes of a warp read different radii, faces and points,
// which a kernel parameter serves one address at a time
template <class Real>
struct MoodW {
  Real z[4][4][kMaxQ][kMaxN];
};
template <class Real>
__device__ __forceinline__ void stage_mood_weights(const DirectW<Real>& Wd, MoodW<Real>& S) {
  Real* zs = &S.z[0][0][0][0];
  const Real* zd = &Wd.z[0][0][0][0];
  for (int k = threadIdx.x; k < 4 * 4 * kMaxQ * kMaxN; k += blockDim.x) zs[k] = zd[k];
  __syncthreads();
}

// entry k (0 itself, 1 W, 2 E, 3 S, 4 N) of queued cell c's neighbourhood:
// if c is the first queued cell of that cell's own list (itself, W, E, S,
// N), re-update it, re-detect it and return whether it is troubled; d gets
// the cell's index (or -1)
template <class Real>
__device__ __forceinline__ bool mood_update_item(const StageArgs<Real>& A, const Grid& g,
                                                 const Detect& D, const DirectW<Real>& Wd,
                                                 const Real* d2x, const Real* d2y,
                                                 const uint32_t* stamp, uint32_t cur, int c,
                                                 int k, int& d) {
  const int i = c % g.nx, j = c / g.nx;
  d = k == 0 ? c : neighbour(g, i, j, k - 1);
  if (d < 0) return false;
  const int di = d % g.nx, dj = d / g.nx;
  // the loads of the ownership test and of the candidate depend on d alone:
  // all are issued before the test, so that one memory latency covers them
  bool taken = false;  // cell d is updated by another queued cell's item
  if (k > 0) {
    taken = stamp[d] == cur;
    // earlier entries of d's own list: W, E, S (in that order) before c
    const int back = k == 1 ? 1 : k == 2 ? 0 : k == 3 ? 3 : 2;
    for (int e = 0; e < 3; ++e) {
      if (e >= back) break;
      int o = neighbour(g, di, dj, e);
      taken |= o >= 0 && stamp[o] == cur;
    }
  }
  double Y[4];
  candidate<Real>(A, g, di, dj, A.sc->dt, Y);
  const int od = A.ord[d];
  if (taken) {
    d = -1;
    return false;
  }
  bool flag = false;
  if (od != 0) {
    flag = face_state_bad<Real>(A, g, di, dj) ||
           troubled_prefetched<Real>(A.Xr, g, D, d2x, d2y, di, dj, Y);
  } else {
    Real y[4] = {(Real)Y[0], (Real)Y[1], (Real)Y[2], (Real)Y[3]};
    Real p = (Real)(g.gamma - 1.0) * (y[3] - Real(0.5) * (y[1] * y[1] + y[2] * y[2]) / y[0]);
    if (!(y[0] > Real(0)) || !(p > Real(0))) atomicAdd(&A.scw->nfog_pad[A.stage], 1);
  }
  combine_store<Real>(A, g, di, dj, Y);
  return flag;
}

// ---------------------------------------------------------------------------
// the whole MOOD loop of one stage in one cooperative launch (Sec. 4 Step 10:
// repeat until no cell is flagged).  Every block takes part in every phase of
// every iteration, separated by grid-wide barriers:
//   lower the queued cells one cascade level  | barrier
//   recompute the faces whose EDP1 radius changed  | barrier
//   re-update + re-detect the queued cells and their face neighbours,
//   troubled ones into the other queue  | barrier
// and every block reads the new queue length to take the same decision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// grid-wide barrier of a co-resident grid: the last block to arrive resets
// the count and opens the next generation.  A wait gives up after about a
// second (or 2^26 polls), latches kErrSync and returns false; a block that
// sees the error leaves the loop, so no wait can outlast the limit.
__device__ __forceinline__ bool grid_barrier(Scalars* sc) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &sc->bar_gen;
    volatile int* err = &sc->err;
    const unsigned g0 = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(&sc->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&sc->bar_count, 0u);
      __threadfence();
      atomicAdd(&sc->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (*gen == g0) {
        if (++polls > (1u << 26) || global_ns() - t0 > 1000000000ull) {
          atomicOr(&sc->err, kErrSync);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
    }
    if (*err & kErrSync) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// the stamps of value v: two arrays, one per parity of v, so that an
// iteration can mark the cells of the next queue (value v + 1) while its own
// queue's marks (value v) are still being read
__device__ __forceinline__ uint32_t* stamp_of(const MoodArgs& M, uint32_t v) {
  return M.stamp + (long long)(v & 1u) * M.stamp_stride;
}

// problem of a pooled cell index gc: the handle's single problem
template <class Real>
struct SingleSite {
  const StageArgs<Real>& A;
  const Grid& g;
  const Detect& D;
  const Real* d2x;
  const Real* d2y;
  template <class F>
  __device__ __forceinline__ void with(int gc, F&& f) const {
    f(A, g, D, d2x, d2y, 0);
  }
};

// lane index of a MOOD phase: the warps are ranked block-minor (warp 0 of
// every block, then warp 1, ...), so the few warps of a short iteration land
// on different SMs and FP64 sub-partitions instead of queueing on one
__device__ __forceinline__ long long mood_lane() {
  return ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}

// the MOOD face recompute with one lane per Gauss point: lane t covers
// pooled cell queue[t / 16], face (t / 4) % 4, point t % 4.  Each lane
// reconstructs its point's two states and solves its Riemann problem; the
// group's first lane forms the Gauss sum in the order of face_at (mirror
// pairs summed first), so the flux is the same bit for bit.  Called by whole
// warps (the loop runs per warp: all 32 lanes take part in the shuffles).
template <class Real, class Site>
__device__ __forceinline__ void mood_faces_phase(const Site& site, const MoodArgs& M,
                                                 const DirectW<Real>& Wd, const MoodW<Real>& MW,
                                                 const Cascade& C, uint32_t cur,
                                                 const int* queue, int n) {
  const long long L = 16LL * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int base = lane & ~3;
  const uint32_t* stamp = stamp_of(M, cur);
  for (long long t0 = mood_lane() - lane; t0 < L; t0 += stride) {
    const long long t = t0 + lane;
    const int q = (int)(t & 3);
    const int f = (int)((t >> 2) & 3);
    const int gc = t < L ? queue[t >> 4] : 0;
    int iL = 0, jL = 0, K = 0;
    bool work = false;
    Real fq[4] = {Real(0), Real(0), Real(0), Real(0)};
    bool bl = false, br = false;
    if (t < L)
      site.with(gc, [&](const StageArgs<Real>& A, const Grid& g, const Detect&, const Real*,
                        const Real*, int off) {
        work = mood_face_plan<Real>(A, g, C, stamp + off, cur, gc - off, f, iL, jL, K);
        if (work && q < rule_q(K)) {
          // a recorded step keeps the states of the recomputed face
          const bool keep = A.sc->ctl.stape != nullptr;
          Real UL[4], UR[4];
          const int dir = f < 2 ? 0 : 1;
          if constexpr (sizeof(Real) == sizeof(double))
            face_point_rt<Real>(K, dir, A.Xr, g, MW.z[K][2 * dir][q], MW.z[K][2 * dir + 1][q],
                                iL, jL, fq, bl, br, keep ? UL : nullptr, UR);
          else if (dir == 0)
            face_point_k<Real, 0>(K, A.Xr, g, Wd, iL, jL, q, fq, bl, br, keep ? UL : nullptr, UR);
          else
            face_point_k<Real, 1>(K, A.Xr, g, Wd, iL, jL, q, fq, bl, br, keep ? UL : nullptr, UR);
          if (keep) {
            const int qt = rule_q(Wd.top);
            if (f < 2) tape_face<Real, 0>(A, g, qt, iL, jL, q, UL, UR);
            else tape_face<Real, 1>(A, g, qt, iL, jL, q, UL, UR);
          }
        }
      });
    Real fp[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int v = 0; v < 4; ++v) fp[p][v] = __shfl_sync(0xffffffffu, fq[v], base + p);
    const unsigned bbl = __ballot_sync(0xffffffffu, bl), bbr = __ballot_sync(0xffffffffu, br);
    if (work && q == 0) {
      // face_at's loop over (g, -g) pairs, one path for every rule size:
      // Q = 4: w1 (f1 + f2) + w0 (f0 + f3); Q = 3: w1 f1 + w0 (f0 + f2);
      // Q = 2: w0 (f0 + f1); Q = 1: w0 (f0 + 0), which rounds as w0 f0
      const int Q = rule_q(K);
      const Real w0 = Wd.w[K][0], w1 = Wd.w[K][1];
      Real F[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const Real z = Real(0);
        const Real last = Q == 4 ? fp[3][v] : Q == 3 ? fp[2][v] : Q == 2 ? fp[1][v] : z;
        const Real inner = fma(w0, add_rn(fp[0][v], last), z);
        const Real mid = Q == 4 ? add_rn(fp[1][v], fp[2][v]) : fp[1][v];
        const Real outer = fma(w1, mid, inner);
        F[v] = Q >= 3 ? outer : inner;
      }
      const uint8_t bits = (uint8_t)((((bbl >> base) & 0xFu) ? 1 : 0) |
                                     (((bbr >> base) & 0xFu) ? 2 : 0));
      site.with(gc, [&](const StageArgs<Real>& A, const Grid& g, const Detect&, const Real*,
                        const Real*, int) {
        if (f < 2) store_face<Real, 0>(A, g, iL, jL, F, bits);
        else store_face<Real, 1>(A, g, iL, jL, F, bits);
      });
    }
  }
}

// re-update + re-detect: item t is entry t % 5 (itself, W, E, S, N) of
// pooled cell queue[t / 5]; a cell found troubled is lowered one cascade
// level at once, marked with the next stamp and appended to the next queue
template <class Real, class Site>
__device__ __forceinline__ void mood_update_phase(const Site& site, const MoodArgs& M,
                                                  const DirectW<Real>& Wd, const Cascade& C,
                                                  uint32_t cur, const int* queue, int n,
                                                  int* next_queue, int* next_count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const uint32_t* stamp = stamp_of(M, cur);
  uint32_t* next_stamp = stamp_of(M, cur + 1);
  for (long long t = mood_lane(); t < 5LL * n; t += stride) {
    const int gc = queue[t / 5];
    int dg = -1;
    bool flag = false;
    site.with(gc, [&](const StageArgs<Real>& A, const Grid& g, const Detect& D, const Real* d2x,
                      const Real* d2y, int off) {
      int d = -1;
      flag = mood_update_item<Real>(A, g, D, Wd, d2x, d2y, stamp + off, cur, gc - off,
                                    (int)(t % 5), d);
      if (flag) {
        // only this item updates cell d in this iteration: its radius and
        // its next stamp are written by no one else
        A.ord[d] = (uint8_t)C.next[A.ord[d]];
        next_stamp[off + d] = cur + 1;
      }
      dg = d >= 0 ? off + d : -1;
    });
    queue_push(flag, dg, next_queue, next_count);
  }
}

// the loop itself, for one problem or a batch (Site).  The first-pass queue
// is lowered and marked in a prologue; then every iteration is
//   recompute the faces whose EDP1 radius changed  | barrier
//   re-update + re-detect, lowering and marking the troubled cells
//   for the next iteration  | barrier
// and every block reads the new queue length to take the same decision.
template <class Real, class Site>
__device__ __forceinline__ void mood_loop_body(const Site& site, const MoodArgs& M,
                                               const DirectW<Real>& Wd, const Cascade& C,
                                               int stage) {
  Scalars* sc = M.sc;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // the first pass filled queue 0; queue 1 receives the first iteration's
  // troubled cells (its count is cleared here, read after two barriers)
  int n = *(volatile int*)&sc->count[0];
  const int nfirst = n;
  int slot = 0, iters = 0, total = n;
  uint32_t cur = sc->stamp_cur + 1;  // stamp of the cells of the first queue
  const int cap = sc->ctl.max_iters;
  if (leader) sc->count[1] = 0;
  bool ok = true;
  __shared__ MoodW<Real> MW;
  if (n > 0) {
    // n is the same in every block; FP32 reads the kernel parameter
    if constexpr (sizeof(Real) == sizeof(double)) stage_mood_weights<Real>(Wd, MW);
    uint32_t* st = stamp_of(M, cur);
    for (long long q = mood_lane(); q < n; q += stride) {
      const int gc = M.queue[0][q];
      site.with(gc, [&](const StageArgs<Real>& A, const Grid&, const Detect&, const Real*,
                        const Real*, int off) {
        A.ord[gc - off] = (uint8_t)C.next[A.ord[gc - off]];
      });
      st[gc] = cur;
    }
    ok = grid_barrier(sc);
  }
  while (ok && n > 0) {
    if (iters >= cap) {
      if (leader) atomicOr(&sc->err, kErrCap);
      break;
    }
    const int* queue = M.queue[slot];
    mood_faces_phase<Real>(site, M, Wd, MW, C, cur, queue, n);
    if (!grid_barrier(sc)) break;
    int* next_count = &sc->count[slot ^ 1];
    mood_update_phase<Real>(site, M, Wd, C, cur, queue, n, M.queue[slot ^ 1], next_count);
    if (!grid_barrier(sc)) break;
    n = *(volatile int*)next_count;
    // the queue just worked on receives the next iteration's cells
    if (leader) sc->count[slot] = 0;
    total += n;
    iters += 1;
    slot ^= 1;
    cur += 1;
  }
  if (leader) {
    sc->nbad_first[stage] = nfirst;
    sc->nbad_total[stage] = total;
    sc->iters[stage] = iters;
    sc->stamp_cur = cur;  // every value up to cur has been used
    sc->slot = 0;
    sc->go = 0;
    // both queues empty for the next stage, also after a failed loop
    sc->count[0] = 0;
    sc->count[1] = 0;
  }
}

// the loop's tail (LoopTail): every interior value of the stage output is
// final once the loop has ended (the last phase ended at a grid barrier, or
// the first pass, a previous kernel, wrote them all)
__device__ __forceinline__ void mood_loop_tail(const Grid& g, Scalars* sc, const LoopTail& T) {
  const long long tid = ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 +
                        (threadIdx.x & 31);
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (T.X) {
    const double t = sc->t + T.tfrac * sc->dt;
    const long long n = ghost_count(g);
    for (long long k = tid; k < n; k += stride) fill_ghost(T.X, T.Xf, g, t, k);
  }
  if (T.rate) {
    // as k_dt_reduce, for the next step: the maximum CFL rate over the cells
    double best = 0.0;
    bool bad = false;
    const long long n = (long long)g.nx * g.ny;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
      const int i = (int)(c % g.nx), j = (int)(c / g.nx);
      double a;
      if (!cell_rate_at(T.Xrate, T.Xfrate, g, i, j, a)) bad = true;
      else best = max_num(a, best);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && g.rate_floor > best) best = g.rate_floor;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = max_num(ob, best);
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
      if (bad) atomicOr(&sc->rate_bad, 1);
      if (best > 0.0) atomicMax(&sc->rate_bits, (unsigned long long)__double_as_longlong(best));
    }
    // readers are later kernels: the flag can go up before every block is done
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->rate_ready = 1;
  }
}

template <class Real>
__global__ void __launch_bounds__(256, 2) k_mood_loop(StageArgs<Real> A, MoodArgs M, Grid g,
                                                   Detect D,
                                                   const __grid_constant__ DirectW<Real> Wd,
                                                   Cascade C, int stage, LoopTail T) {
  pdl_wait();
  const SingleSite<Real> site{A, g, D, Wd.d2x, Wd.d2y};
  mood_loop_body<Real>(site, M, Wd, C, stage);
  mood_loop_tail(g, M.sc, T);
}

// ---------------------------------------------------------------------------
// replay of a step with given radii (no detection): every face at the EDP1
// radius of a radius map, then candidate + RK combination
// ---------------------------------------------------------------------------
template <class Real, int DIR>
__global__ void __launch_bounds__(128) k_faces_frozen(StageArgs<Real> A, Grid g,
                                                      const __grid_constant__ DirectW<Real> Wd) {
  const long long nf = DIR == 0 ? (long long)(g.nx + 1) * g.ny : (long long)g.nx * (g.ny + 1);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int iL, jL;
  if (DIR == 0) {
    iL = (int)(f % (g.nx + 1)) - 1;
    jL = (int)(f / (g.nx + 1));
  } else {
    iL = (int)(f % g.nx);
    jL = (int)(f / g.nx) - 1;
  }
  const int iR = iL + (DIR == 0), jR = jL + (DIR == 1);
  auto rad = [&](int i, int j) -> int {
    if (i < 0 || i >= g.nx) {
      if (!g.periodic_x) return Wd.top;
      i = wrapi(i, g.nx);
    }
    if (j < 0 || j >= g.ny) {
      if (!g.periodic_y) return Wd.top;
      j = wrapi(j, g.ny);
    }
    return A.ord[cidx(g, i, j)];
  };
  const int a = rad(iL, jL), b = rad(iR, jR);
  const int K = a < b ? a : b;
  Real F[4];
  bool bl, br;
  switch (K) {
    case 0: face_at<0, Real, DIR>(A.Xr, g, Wd, iL, jL, F, bl, br); break;
    case 1: face_at<1, Real, DIR>(A.Xr, g, Wd, iL, jL, F, bl, br); break;
    case 2: face_at<2, Real, DIR>(A.Xr, g, Wd, iL, jL, F, bl, br); break;
    default: face_at<3, Real, DIR>(A.Xr, g, Wd, iL, jL, F, bl, br); break;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (DIR == 0) A.Fx[fxidx(g, v, iR, jL)] = F[v];
    else A.Fy[fyidx(g, v, iL, jR)] = F[v];
  }
}

template <class Real>
__global__ void __launch_bounds__(256) k_update_frozen(StageArgs<Real> A, Grid g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  double Y[4];
  candidate<Real>(A, g, i, j, A.sc->dt, Y);
  combine_store<Real>(A, g, i, j, Y);
}

// ---------------------------------------------------------------------------
// batched kernels: many independent problems of uneven sizes in one
// persistent launch per kernel class.  Each block walks a list of work items
// (problem, block coordinates); the problem's grid is staged in shared
// memory; all buffers are pooled, each problem at its own offsets.  A
// problem with dt = 0 (finished) only carries its state over.
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ StageArgs<Real> problem_args(const StageArgs<Real>& B, const Prob& P,
                                                        const Scalars* psc, int p) {
  StageArgs<Real> A = B;
  A.X = B.X + P.state_off;
  A.Xr = B.Xr + P.state_off;
  A.U0 = B.U0 + P.state_off;
  A.out = B.out + P.state_off;
  A.outr = B.outr ? B.outr + P.state_off : nullptr;
  A.W = B.W ? B.W + P.state_off : nullptr;
  A.out2 = B.out2 ? B.out2 + P.state_off : nullptr;
  A.Fx = B.Fx + P.fx_off;
  A.Fy = B.Fy + P.fy_off;
  A.fbx = B.fbx + P.fx_off / 4;  // face planes: one per variable in the flux pools
  A.fby = B.fby + P.fy_off / 4;
  A.ord = B.ord + P.cell_off;
  A.first = B.first + P.cell_off;
  A.sc = psc + p;
  return A;
}

template <class Real>
__device__ __forceinline__ const Real* d2_of(const Prob& P, int d);
template <>
__device__ __forceinline__ const double* d2_of<double>(const Prob& P, int d) {
  return d == 0 ? P.d2x : P.d2y;
}
template <>
__device__ __forceinline__ const float* d2_of<float>(const Prob& P, int d) {
  return d == 0 ? P.d2xf : P.d2yf;
}

// one block per work item: a software loop over items would let the
// compiler keep all parity weights in registers across items (they are loop
// invariant), doubling the register footprint; the block scheduler walks the
// item list instead
template <int R, class Real, int DIR, int FW>
__global__ void __launch_bounds__(32 * FW) k_faces_batch(StageArgs<Real> B, const Prob* probs,
                                                         const Scalars* psc, const Item* items,
                                                         const __grid_constant__ ParityW<Real> W) {
  pdl_wait();
  pdl_trigger();
  __shared__ FaceTile<R, Real, FW> tile;
  // the item's problem, read from shared memory on demand like kernel
  // parameters
  __shared__ Prob sp;
  __shared__ StageArgs<Real> sa;
  __shared__ int sw[3];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const Item w = items[blockIdx.x];
    sp = probs[w.p];
    sa = problem_args<Real>(B, sp, psc, w.p);
    sw[0] = psc[w.p].dt == 0.0;  // finished problem
    sw[1] = w.a;
    sw[2] = w.b;
  }
  __syncthreads();
  if (sw[0]) return;  // uniform over the block
  faces_block<R, Real, DIR, FW>(sa, sp.g, W, sw[1], sw[2], tile);
}

// the fused x+y face kernel over (problem, segment, band) work items
template <int R, class Real>
__global__ void __launch_bounds__(32 * kXYRows, xy_min_blocks<Real>()) k_faces_xy_batch(
    StageArgs<Real> B, const Prob* probs, const Scalars* psc, const Item* items,
    const __grid_constant__ ParityW<Real> W) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char xy_smem[];
  XYShared<R, Real>& S = *reinterpret_cast<XYShared<R, Real>*>(xy_smem);
  __shared__ Prob sp;
  __shared__ StageArgs<Real> sa;
  __shared__ int sw[3];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const Item w = items[blockIdx.x];
    sp = probs[w.p];
    sa = problem_args<Real>(B, sp, psc, w.p);
    sw[0] = psc[w.p].dt == 0.0;  // finished problem
    sw[1] = w.a;
    sw[2] = w.b;
  }
  __syncthreads();
  if (sw[0]) return;  // uniform over the block
  faces_xy_block<R, Real>(sa, sp.g, W, sw[1], sw[2], S);
}

template <class Real>
__global__ void __launch_bounds__(256) k_update_batch(StageArgs<Real> B, const Prob* probs,
                                                      const Scalars* psc, const Item* items,
                                                      int nitems,
                                                      const __grid_constant__ DirectW<Real> Wd) {
  __shared__ Prob sp;
  __shared__ StageArgs<Real> sa;
  __shared__ StageC sk;
  __shared__ int sw[3];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    __syncthreads();
    if (tid == 0) {
      const Item w = items[it];
      sp = probs[w.p];
      sa = problem_args<Real>(B, sp, psc, w.p);
      sw[0] = psc[w.p].dt == 0.0;
      sw[1] = w.a;
      sw[2] = w.b;
      if (!sw[0]) sk = stage_coeffs<Real>(sa, sp.g, sa.sc->dt);
    }
    __syncthreads();
    const int i = sw[1] * 32 + threadIdx.x, j = sw[2] * 8 + threadIdx.y;
    if (sw[0]) {
      // finished: carry the state over unchanged
      if (i < sp.g.nx && j < sp.g.ny) {
#pragma unroll
        for (int v = 0; v < 4; ++v) sa.out[gidx(sp.g, v, i, j)] = sa.X[gidx(sp.g, v, i, j)];
      }
      continue;
    }
    update_cell_w<Real>(sa, sp.g, sp.det, Wd, d2_of<Real>(sp, 0), d2_of<Real>(sp, 1), i, j,
                        sp.cell_off, sk);
  }
}

// problem of a pooled cell index (probs sorted by cell_off)
__device__ __forceinline__ int problem_of(const Prob* probs, int nprob, int gc) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].cell_off <= gc) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// problem of a pooled cell index gc in a batch (problems sorted by their
// first cell)
template <class Real>
struct BatchSite {
  const StageArgs<Real>& B;
  const Prob* probs;
  const Scalars* psc;
  int nprob;
  template <class F>
  __device__ __forceinline__ void with(int gc, F&& f) const {
    const int p = problem_of(probs, nprob, gc);
    const Prob& P = probs[p];
    const StageArgs<Real> A = problem_args<Real>(B, P, psc, p);
    f(A, P.g, P.det, d2_of<Real>(P, 0), d2_of<Real>(P, 1), P.cell_off);
  }
};

template <class Real>
__global__ void __launch_bounds__(256, 2) k_mood_loop_batch(StageArgs<Real> B, MoodArgs M,
                                                         const Prob* probs, const Scalars* psc,
                                                         int nprob,
                                                         const __grid_constant__ DirectW<Real> Wd,
                                                         Cascade C, int stage) {
  const BatchSite<Real> site{B, probs, psc, nprob};
  mood_loop_body<Real>(site, M, Wd, C, stage);
}

}  // namespace gpm
