// weight_tables.h -- kernel weight tables from the binary128 solves: the
// full per-radius prediction vectors for the MOOD recompute and the parity
// coefficients of the top radius for the first pass.
#pragma once

#include <string.h>

#include "gp_weights.h"
#include "gpmood_kernels.cuh"

namespace gpm {
namespace {

// index of offset (a,b) in the stencil order of gp_weights.c
int sidx(const gpw_radius& w, int a, int b) {
  for (int m = 0; m < w.n; ++m)
    if (w.da[m] == a && w.db[m] == b) return m;
  return -1;
}

template <class Real>
void fill_weights(const gpw_radius* wr, int top, const double* d2x, const double* d2y,
                  ParityW<Real>& P, DirectW<Real>& D) {
  memset(&P, 0, sizeof(P));
  memset(&D, 0, sizeof(D));
  D.top = top;
  D.w[0][0] = Real(1);
  for (int m = 0; m < 5; ++m) {
    D.d2x[m] = (Real)d2x[m];
    D.d2y[m] = (Real)d2y[m];
  }
  for (int R = 1; R <= 3; ++R) {
    const gpw_radius& w = wr[R];
    if (w.n == 0) continue;
    const int q = w.q;
    for (int k = 0; k < q; ++k) D.w[R][k] = (Real)w.w[k];
    // direct weights from the east / north solves at g >= 0 by the mirrors
    for (int k = 0; k < q; ++k) {
      const int kp = k < (q + 1) / 2 ? k : q - 1 - k;  // the +g point of the pair
      const bool neg = k != kp;
      for (int m = 0; m < w.n; ++m) {
        int a = w.da[m], b = w.db[m];
        // E at g: z_E(g)(a,b); E at -g: z_E(g)(a,-b); W: x-mirror of E
        D.z[R][0][k][m] = (Real)w.z[0][kp][sidx(w, a, neg ? -b : b)];
        D.z[R][1][k][m] = (Real)w.z[0][kp][sidx(w, -a, neg ? -b : b)];
        // N at g: z_N(g)(a,b); N at -g: z_N(g)(-a,b); S: y-mirror of N
        D.z[R][2][k][m] = (Real)w.z[1][kp][sidx(w, neg ? -a : a, b)];
        D.z[R][3][k][m] = (Real)w.z[1][kp][sidx(w, neg ? -a : a, -b)];
      }
    }
  }
  // parity coefficients of the top radius
  const int R = top;
  if (R == 0) {
    P.cx[0][0] = P.cy[0][0] = Real(1);
    P.w[0] = Real(1);
    return;
  }
  const gpw_radius& w = wr[R];
  const int q = w.q, ns = (q + 1) / 2;
  for (int k = 0; k < q; ++k) P.w[k] = (Real)w.w[k];
  for (int kk = 0; kk < ns; ++kk) {
    const bool middle = (q & 1) && kk == q / 2;
    for (int c = 0; c < stencil_n(R); ++c) {
      Comp cm = comp_at(R, c);
      double ex = 0.0, ny = 0.0;
      int cnt = 0;
      for (int sa = 1; sa >= -1; sa -= 2) {
        if (cm.a == 0 && sa < 0) continue;
        for (int sb = 1; sb >= -1; sb -= 2) {
          if (cm.b == 0 && sb < 0) continue;
          double chi = (cm.px && sa < 0 ? -1.0 : 1.0) * (cm.py && sb < 0 ? -1.0 : 1.0);
          ex += chi * w.z[0][kk][sidx(w, sa * cm.a, sb * cm.b)];
          ny += chi * w.z[1][kk][sidx(w, sa * cm.a, sb * cm.b)];
          ++cnt;
        }
      }
      ex /= cnt;
      ny /= cnt;
      // at g = 0 the odd components across the face vanish exactly
      if (middle && cm.py) ex = 0.0;
      if (middle && cm.px) ny = 0.0;
      P.cx[kk][c] = (Real)ex;
      P.cy[kk][c] = (Real)ny;
    }
  }
}

}  // namespace
}  // namespace gpm
