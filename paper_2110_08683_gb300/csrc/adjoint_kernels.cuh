// adjoint_kernels.cuh -- reverse mode of one SSP-RK3 step with the GP radii
// of every stage and the time step held at their forward values.
//
// For a stage Y = X - dt F(X) the vector-Jacobian product is
//   v^T dY/dX = v - dt (dF/dX)^T v,
// and (dF/dX)^T v is formed in three passes:
//   1. faces: the adjoint of the face-averaged flux of eq. fvm_F is
//      a_f = (v_L - v_R)/dx (or /dy); at every Gauss point of the face's EDP1
//      radius the states are reconstructed again and the HLLC flux is
//      differentiated in reverse (w_g a_f in, state adjoints out);
//   2. gather: every cell of the ghosted grid collects z_m times the state
//      adjoints of the faces whose reconstruction stencil contains it
//      (eq. gp_reconstructor transposed);
//   3. fold: ghost-cell adjoints go back to the interior cells the ghosts
//      copied (periodic wrap-add, outflow add, reflect with the normal
//      momentum negated, fixed states drop out).
#pragma once

#include "gpmood_kernels.cuh"

namespace gpm {

// x != 0 as IEEE decides it (a NaN is nonzero), on the integer pipes in FP64
__device__ __forceinline__ bool nonzero(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ bool nonzero(float x) { return x != 0.0f; }

// inverse square root by Newton-Raphson from the hardware approximation:
// each step y <- y (3/2 - (z/2) y^2) squares the relative error.  FP64:
// rsqrt.approx.ftz.f64 and two steps; FP32: rsqrt.approx.ftz.f32 and one.
__device__ __forceinline__ double rsqrt_nr(double z) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(z));
  const double h = 0.5 * z;
  y = y * fma(-h * y, y, 1.5);
  return y * fma(-h * y, y, 1.5);
}
__device__ __forceinline__ float rsqrt_nr(float z) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(z));
  return y * fmaf(-0.5f * z * y, y, 1.5f);
}

// reverse mode of hllc_x: given the adjoint Fb of the flux, accumulate the
// adjoints of the two states into UbL / UbR.  The forward expressions are
// those of hllc_x (the same algebra; the sound speed as z / sqrt(z), whose
// derivative 1 / (2 sqrt(z)) comes with it); only the branch the forward
// took is differentiated.
template <class Real>
__device__ __forceinline__ void hllc_x_vjp(const Real* UL, const Real* UR, Real gam,
                                           const Real* Fb, Real* UbL, Real* UbR) {
  const Real gm1 = gam - Real(1);
  // ---- forward, keeping the intermediates
  const Real rL = UL[0], rR = UR[0];
  const Real irL = recip(rL), irR = recip(rR);
  const Real uL = UL[1] * irL, vL = UL[2] * irL;
  const Real uR = UR[1] * irR, vR = UR[2] * irR;
  const Real pL = gm1 * (UL[3] - Real(0.5) * (UL[1] * uL + UL[2] * vL));
  const Real pR = gm1 * (UR[3] - Real(0.5) * (UR[1] * uR + UR[2] * vR));
  const Real zL = gam * pL * irL, zR = gam * pR * irR;
  const Real yL = rsqrt_nr(zL), yR = rsqrt_nr(zR);  // 1 / c
  const Real cL = zL * yL, cR = zR * yR;
  const Real aL = uL - cL, bL = uR - cR;
  const bool selA = lt_num(aL, bL);
  const Real SL = selA ? aL : bL;
  const Real aR = uL + cL, bR = uR + cR;
  const bool selAR = lt_num(bR, aR);
  const Real SR = selAR ? aR : bR;
  const Real dL = SL - uL, dR = SR - uR;
  const Real num = pR - pL + rL * uL * dL - rR * uR * dR;
  const Real den = rL * dL - rR * dR;
  const Real iden = recip(den);
  const Real Ss = num * iden;
  // the forward's decisions, compared on the integer pipes (the taped
  // states lie in the solver's domain, where every value is finite)
  const bool left = ge0_num(Ss);
  const bool useL = ge0_num(SL);
  const bool useS = !useL && (left || gt0_num(SR));
  // the one physical flux the forward used: F_L if S_L >= 0, F_R if
  // S_R <= 0, else F_K of the star side; its adjoint is Fb in every case
  const bool sideL = useL || (useS && left);
  // adjoints of the intermediates
  Real rLb = 0, rRb = 0, uLb = 0, uRb = 0, vLb = 0, vRb = 0, pLb = 0, pRb = 0, ELb = 0, ERb = 0;
  Real SLb = 0, SRb = 0, Ssb = 0, irLb = 0, irRb = 0, dLb = 0, dRb = 0;
  if (useS) {
    // star state of side K (hllc_x's second form: m = rho_K d_K,
    // D = 1 / (S_K - S*), rho* = m D, (rho E)* = D (d_K E_K + (S* - u_K) A),
    // A = m S* + p_K)
    const Real rK = left ? rL : rR, uK = left ? uL : uR, vK = left ? vL : vR;
    const Real EK = left ? UL[3] : UR[3], pK = left ? pL : pR, SK = left ? SL : SR;
    const Real dK = left ? dL : dR;
    const Real iD = recip(SK - Ss);
    const Real m = rK * dK;
    const Real fK = m * iD;
    const Real t1 = Ss - uK, Aq = m * Ss + pK;
    const Real Cq = dK * EK + t1 * Aq;
    const Real UKs[4] = {fK, fK * Ss, fK * vK, iD * Cq};
    const Real* UK = left ? UL : UR;
    // Fs[v] = FK[v] + SK (UKs[v] - UK[v])
    Real UKsb[4], SKb = 0, UKb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      SKb += Fb[k] * (UKs[k] - UK[k]);
      UKsb[k] = SK * Fb[k];
      UKb[k] = -SK * Fb[k];
    }
    // UKs = (fK, fK Ss, fK vK, iD Cq), fK = m iD
    Real fKb = UKsb[0] + UKsb[1] * Ss + UKsb[2] * vK;
    Ssb += UKsb[1] * fK;
    Real vKb = UKsb[2] * fK;
    const Real Cb = UKsb[3] * iD;
    Real iDb = UKsb[3] * Cq + fKb * m;
    // Cq = dK EK + t1 Aq, t1 = Ss - uK, Aq = m Ss + pK
    Real dKb = Cb * EK;
    Real EKb = Cb * dK;
    const Real Ab = Cb * t1;
    Ssb += Cb * Aq;
    Real uKb = -Cb * Aq;
    Real pKb = Ab;
    const Real mb = Ab * Ss + fKb * iD;
    Ssb += Ab * m;
    // m = rK dK
    Real rKb = mb * dK;
    dKb += mb * rK;
    // iD = 1 / D, D = SK - Ss
    const Real Db = -iDb * iD * iD;
    SKb += Db;
    Ssb -= Db;
    if (left) {
      rLb += rKb; uLb += uKb; vLb += vKb; ELb += EKb; pLb += pKb; SLb += SKb;
      dLb += dKb;
#pragma unroll
      for (int k = 0; k < 4; ++k) UbL[k] += UKb[k];
    } else {
      rRb += rKb; uRb += uKb; vRb += vKb; ERb += EKb; pRb += pKb; SRb += SKb;
      dRb += dKb;
#pragma unroll
      for (int k = 0; k < 4; ++k) UbR[k] += UKb[k];
    }
    // Ss = num / den
    const Real numb = Ssb * iden;
    const Real denb = -Ssb * Ss * iden;
    // den = rL dL - rR dR
    rLb += denb * dL; dLb += denb * rL; rRb -= denb * dR; dRb -= denb * rR;
    // num = pR - pL + rL uL dL - rR uR dR
    pRb += numb; pLb -= numb;
    rLb += numb * uL * dL; uLb += numb * rL * dL; dLb += numb * rL * uL;
    rRb -= numb * uR * dR; uRb -= numb * rR * dR; dRb -= numb * rR * uR;
  }
  // dL = SL - uL, dR = SR - uR
  SLb += dLb; uLb -= dLb;
  SRb += dRb; uRb -= dRb;
  // SL = min(aL, bL), SR = max(aR, bR) on the branch taken
  Real cLb = 0, cRb = 0;
  if (selA) { uLb += SLb; cLb -= SLb; } else { uRb += SLb; cRb -= SLb; }
  if (selAR) { uLb += SRb; cLb += SRb; } else { uRb += SRb; cRb += SRb; }
  // the physical flux of side X, F = (r u, r u u + p, r u v, u (E + p))
  {
    const Real rX = sideL ? rL : rR, uX = sideL ? uL : uR, vX = sideL ? vL : vR;
    const Real pX = sideL ? pL : pR, EX = sideL ? UL[3] : UR[3];
    const Real rXb = Fb[0] * uX + Fb[1] * uX * uX + Fb[2] * uX * vX;
    const Real uXb = Fb[0] * rX + Fb[1] * Real(2) * rX * uX + Fb[2] * rX * vX + Fb[3] * (EX + pX);
    const Real vXb = Fb[2] * rX * uX, pXb = Fb[1] + Fb[3] * uX, EXb = Fb[3] * uX;
    if (sideL) {
      rLb += rXb; uLb += uXb; vLb += vXb; pLb += pXb; ELb += EXb;
    } else {
      rRb += rXb; uRb += uXb; vRb += vXb; pRb += pXb; ERb += EXb;
    }
  }
  // c = sqrt(z), z = gam p ir: dc/dz = 1 / (2 c) = y / 2
  const Real zLb = cLb * Real(0.5) * yL, zRb = cRb * Real(0.5) * yR;
  if (nonzero(cLb)) { pLb += zLb * gam * irL; irLb += zLb * gam * pL; }
  if (nonzero(cRb)) { pRb += zRb * gam * irR; irRb += zRb * gam * pR; }
  // p = gm1 (E - 0.5 (m_x u + m_y v))
  ELb += pLb * gm1;
  Real mxLb = -Real(0.5) * gm1 * pLb * uL, myLb = -Real(0.5) * gm1 * pLb * vL;
  uLb -= Real(0.5) * gm1 * pLb * UL[1];
  vLb -= Real(0.5) * gm1 * pLb * UL[2];
  ERb += pRb * gm1;
  Real mxRb = -Real(0.5) * gm1 * pRb * uR, myRb = -Real(0.5) * gm1 * pRb * vR;
  uRb -= Real(0.5) * gm1 * pRb * UR[1];
  vRb -= Real(0.5) * gm1 * pRb * UR[2];
  // u = m_x ir, v = m_y ir
  mxLb += uLb * irL; myLb += vLb * irL; irLb += uLb * UL[1] + vLb * UL[2];
  mxRb += uRb * irR; myRb += vRb * irR; irRb += uRb * UR[1] + vRb * UR[2];
  // ir = 1 / r
  rLb -= irLb * irL * irL;
  rRb -= irRb * irR * irR;
  UbL[0] += rLb; UbL[1] += mxLb; UbL[2] += myLb; UbL[3] += ELb;
  UbR[0] += rRb; UbR[1] += mxRb; UbR[2] += myRb; UbR[3] += ERb;
}

// EDP1 radius of the face between (iL,jL) and (iR,jR) from a radius map
__device__ __forceinline__ int face_radius(const Grid& g, const uint8_t* ord, int top, int iL,
                                           int jL, int iR, int jR) {
  auto rad = [&](int i, int j) -> int {
    if (i < 0 || i >= g.nx) {
      if (!g.periodic_x) return top;
      i = wrapi(i, g.nx);
    }
    if (j < 0 || j >= g.ny) {
      if (!g.periodic_y) return top;
      j = wrapi(j, g.ny);
    }
    return ord[cidx(g, i, j)];
  };
  const int a = rad(iL, jL), b = rad(iR, jR);
  return a < b ? a : b;
}

// reverse mode of one Gauss point q of a face: states UL / UR, flux adjoint
// w_q a; the state adjoints go to the face's slots of A.L / A.R
template <class Real, int DIR>
__device__ __forceinline__ void adj_point(const Real* UL, const Real* UR, Real gam, Real w,
                                          const Real* a, int q, Real* AL, Real* AR, long long f,
                                          long long nf) {
  Real bL[4] = {0, 0, 0, 0}, bR[4] = {0, 0, 0, 0};
  if (DIR == 0) {
    Real Fb[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) Fb[v] = w * a[v];
    hllc_x_vjp<Real>(UL, UR, gam, Fb, bL, bR);
  } else {
    // y faces: HLLC on (rho, rho v, rho u, E); the flux comes back swapped
    Real sL[4] = {UL[0], UL[2], UL[1], UL[3]}, sR[4] = {UR[0], UR[2], UR[1], UR[3]};
    Real sFb[4] = {w * a[0], w * a[2], w * a[1], w * a[3]};
    Real tL[4] = {0, 0, 0, 0}, tR[4] = {0, 0, 0, 0};
    hllc_x_vjp<Real>(sL, sR, gam, sFb, tL, tR);
    bL[0] = tL[0]; bL[1] = tL[2]; bL[2] = tL[1]; bL[3] = tL[3];
    bR[0] = tR[0]; bR[1] = tR[2]; bR[2] = tR[1]; bR[3] = tR[3];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    AL[((long long)v * kMaxQ + q) * nf + f] = bL[v];
    AR[((long long)v * kMaxQ + q) * nf + f] = bR[v];
  }
}

// a face of radius K below the top: states by the direct weights
template <int K, class Real, int DIR>
__device__ void adj_face_at(const Real* X, const Grid& g, const DirectW<Real>& Wd, int iL,
                            int jL, const Real* a, Real* AL, Real* AR, long long f,
                            long long nf) {
  constexpr int Q = rule_q(K);
  const int iR = iL + (DIR == 0), jR = jL + (DIR == 1);
  const Real gam = (Real)g.gamma;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    Real UL[4], UR[4];
    if (K == 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        UL[v] = __ldg(X + gidx(g, v, iL, jL));
        UR[v] = __ldg(X + gidx(g, v, iR, jR));
      }
    } else {
      recon_direct<K, Real, Real>(X, g, Wd.z[K][DIR == 0 ? 0 : 2][q], iL, jL, UL);
      recon_direct<K, Real, Real>(X, g, Wd.z[K][DIR == 0 ? 1 : 3][q], iR, jR, UR);
    }
    adj_point<Real, DIR>(UL, UR, gam, Wd.w[K][q], a, q, AL, AR, f, nf);
  }
}

// flux adjoint of the face between (iL,jL) and (iR,jR): (v_L - v_R)/dx (or
// /dy); ghost sides carry none
template <int DIR>
__device__ __forceinline__ void face_cotangent(const double* vin, const Grid& g, int iL, int jL,
                                               int iR, int jR, double* a) {
  const long long nc = (long long)g.nx * g.ny;
  const bool inL = iL >= 0 && iL < g.nx && jL >= 0 && jL < g.ny;
  const bool inR = iR >= 0 && iR < g.nx && jR >= 0 && jR < g.ny;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double vl = inL ? vin[v * nc + cidx(g, iL, jL)] : 0.0;
    const double vr = inR ? vin[v * nc + cidx(g, iR, jR)] : 0.0;
    a[v] = (vl - vr) * (DIR == 0 ? g.inv_dx : g.inv_dy);
  }
}

// pass 1 on the sweep layout of the first-pass face kernel: one warp per
// row (x faces) or column (y faces) of a 31-face segment, the stencils
// staged in shared memory and the top-radius face states formed from the
// parity sums of each cell; faces whose frozen radius is below the top
// reconstruct with the direct weights of their radius
template <int R, class Real, int DIR, int FW>
__global__ void __launch_bounds__(32 * FW) k_adj_faces_sweep(
    const Real* X, const double* vin, const uint8_t* ord, Grid g,
    const __grid_constant__ ParityW<Real> W, const __grid_constant__ DirectW<Real> Wd,
    AdjFaces A) {
  constexpr int Q = rule_q(R);
  __shared__ FaceTile<R, Real, FW> tile;
  const int seg = DIR == 0 ? blockIdx.x : blockIdx.y, band = DIR == 0 ? blockIdx.y : blockIdx.x;
  tile_load<R, Real, DIR, FW>(tile, X, g, seg, band);
  __syncthreads();
  const int lane = threadIdx.x, warp = threadIdx.y;
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
  const int pos = DIR == 0 ? i : j;
  Real SP[Q][4], SM[Q][4];
  tile_face_states<R, Real, DIR, FW>(tile, W, lane + R, warp + R, pos <= nlen, SP, SM);
  Real SL[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) SL[q][v] = __shfl_up_sync(0xffffffffu, SP[q][v], 1);
  if (lane == 0 || pos < 0 || pos > nlen) return;
  // the face between (iL, jL) and (i, j)
  const int iL = DIR == 0 ? i - 1 : i, jL = DIR == 0 ? j : j - 1;
  const long long f = DIR == 0 ? (long long)j * (g.nx + 1) + i : (long long)j * g.nx + i;
  const int K = face_radius(g, ord, R, iL, jL, i, j);
  A.K[f] = (uint8_t)K;
  double ad[4];
  face_cotangent<DIR>(vin, g, iL, jL, i, j, ad);
  const Real a[4] = {(Real)ad[0], (Real)ad[1], (Real)ad[2], (Real)ad[3]};
  Real* AL = (Real*)A.L;
  Real* AR = (Real*)A.R;
  if (K == R) {
    const Real gam = (Real)g.gamma;
#pragma unroll
    for (int q = 0; q < Q; ++q) adj_point<Real, DIR>(SL[q], SM[q], gam, W.w[q], a, q, AL, AR, f, A.nf);
  } else if (K == 0) {
    adj_face_at<0, Real, DIR>(X, g, Wd, iL, jL, a, AL, AR, f, A.nf);
  } else if (K == 1) {
    adj_face_at<(R > 1 ? 1 : 0), Real, DIR>(X, g, Wd, iL, jL, a, AL, AR, f, A.nf);
  } else {
    adj_face_at<(R > 2 ? 2 : 0), Real, DIR>(X, g, Wd, iL, jL, a, AL, AR, f, A.nf);
  }
}

// pass 1 from the face states a recorded step kept (its state tape): one
// thread per face of direction DIR, no reconstruction.  tL / tR: the
// direction's left and right states [4][qt][faces] of the stage.  The states
// are those the forward solved from, so the result equals the sweep's.
template <class Real, int DIR>
__global__ void __launch_bounds__(128, 4) k_adj_faces_stored(
    const Real* tL, const Real* tR, int qt, const double* vin, const uint8_t* ord, Grid g,
    const __grid_constant__ ParityW<Real> W, const __grid_constant__ DirectW<Real> Wd,
    AdjFaces A) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= A.nf) return;
  int i, j;
  if (DIR == 0) {
    i = (int)(f % (g.nx + 1));
    j = (int)(f / (g.nx + 1));
  } else {
    i = (int)(f % g.nx);
    j = (int)(f / g.nx);
  }
  const int iL = DIR == 0 ? i - 1 : i, jL = DIR == 0 ? j : j - 1;
  const int top = Wd.top;
  const int K = face_radius(g, ord, top, iL, jL, i, j);
  A.K[f] = (uint8_t)K;
  double ad[4];
  face_cotangent<DIR>(vin, g, iL, jL, i, j, ad);
  const Real a[4] = {(Real)ad[0], (Real)ad[1], (Real)ad[2], (Real)ad[3]};
  const Real gam = (Real)g.gamma;
  const int Q = rule_q(K);
  for (int q = 0; q < Q; ++q) {
    Real UL[4], UR[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      UL[v] = tL[((long long)v * qt + q) * A.nf + f];
      UR[v] = tR[((long long)v * qt + q) * A.nf + f];
    }
    const Real w = K == top ? W.w[q] : Wd.w[K][q];
    adj_point<Real, DIR>(UL, UR, gam, w, a, q, (Real*)A.L, (Real*)A.R, f, A.nf);
  }
}

// index of offset (a,b) in the radius-K stencil (order b = -K..K, a = -K..K)
__device__ __forceinline__ int stencil_index(int K, int a, int b) {
  int m = 0;
  for (int bb = -K; bb < b; ++bb) m += 2 * (K - (bb < 0 ? -bb : bb)) + 1;
  const int hb = K - (b < 0 ? -b : b);
  return m + a + hb;
}

template <class Real>
__device__ __forceinline__ void gather_face(const DirectW<Real>& Wd, int face, int a, int b,
                                            int K, const Real* S, long long f, long long nf,
                                            Real* acc) {
  const int ab = (a < 0 ? -a : a) + (b < 0 ? -b : b);
  if (ab > K) return;
  if (K == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] += S[(long long)v * kMaxQ * nf + f];
    return;
  }
  const int m = stencil_index(K, a, b);
  const int Q = K + 1;
  for (int q = 0; q < Q; ++q) {
    const Real z = Wd.z[K][face][q][m];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] = fma(z, S[((long long)v * kMaxQ + q) * nf + f], acc[v]);
  }
}

// pass 2: every cell of the ghosted grid collects from the faces whose
// reconstruction stencils contain it
template <class Real>
__global__ void __launch_bounds__(256) k_adj_gather(Grid g, const __grid_constant__ DirectW<Real> Wd,
                                                    AdjFaces Ax, AdjFaces Ay, double* G) {
  const int gx = g.nx + 2 * g.H, gyy = g.ny + 2 * g.H;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)gx * gyy) return;
  const int ci = (int)(t % gx) - g.H, cj = (int)(t / gx) - g.H;
  const int top = Wd.top;
  Real acc[4] = {0, 0, 0, 0};
  const Real* xL = (const Real*)Ax.L;
  const Real* xR = (const Real*)Ax.R;
  const Real* yL = (const Real*)Ay.L;
  const Real* yR = (const Real*)Ay.R;
  for (int b = -top; b <= top; ++b) {
    const int hb = top - (b < 0 ? -b : b);
    for (int a = -hb; a <= hb; ++a) {
      // n = c - (a, b) reconstructs with c at offset (a, b)
      const int ni = ci - a, nj = cj - b;
      if (nj >= 0 && nj < g.ny) {
        if (ni >= -1 && ni <= g.nx - 1) {  // east face of n: x face ni+1, left state
          const long long f = (long long)nj * (g.nx + 1) + ni + 1;
          gather_face<Real>(Wd, 0, a, b, Ax.K[f], xL, f, Ax.nf, acc);
        }
        if (ni >= 0 && ni <= g.nx) {  // west face of n: x face ni, right state
          const long long f = (long long)nj * (g.nx + 1) + ni;
          gather_face<Real>(Wd, 1, a, b, Ax.K[f], xR, f, Ax.nf, acc);
        }
      }
      if (ni >= 0 && ni < g.nx) {
        if (nj >= -1 && nj <= g.ny - 1) {  // north face of n: y face nj+1, lower state
          const long long f = (long long)(nj + 1) * g.nx + ni;
          gather_face<Real>(Wd, 2, a, b, Ay.K[f], yL, f, Ay.nf, acc);
        }
        if (nj >= 0 && nj <= g.ny) {  // south face of n: y face nj, upper state
          const long long f = (long long)nj * g.nx + ni;
          gather_face<Real>(Wd, 3, a, b, Ay.K[f], yR, f, Ay.nf, acc);
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) G[gidx(g, v, ci, cj)] = (double)acc[v];
}

}  // namespace gpm
