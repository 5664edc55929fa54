// common_kernels.cuh -- precision-independent kernels (ghost fill, time step,
// MOOD bookkeeping); included by the host driver only.
#pragma once

#include "gpmood_kernels.cuh"

namespace gpm {

__global__ void k_fill_ghosts(double* X, Grid g, const Scalars* sc, double tfrac) {
  const int H = g.H;
  const int nxg = g.nx + 2 * H;
  const long long nxs = (long long)g.ny * 2 * H;  // x-ghosts of interior rows
  const long long nys = (long long)2 * H * nxg;   // y-ghost rows
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
    double t = sc->t + tfrac * sc->dt;
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
}


__global__ void k_dt_reduce(const double* X, Grid g, Scalars* sc) {
  double best = INFINITY;
  bool bad = false;
  const long long n = (long long)g.nx * g.ny;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx), j = (int)(c / g.nx);
    double S[4];
    load_cell(X, g, i, j, S);
    double r = S[0], u = S[1] / r, v = S[2] / r;
    double p = (g.gamma - 1.0) * (S[3] - 0.5 * (S[1] * S[1] + S[2] * S[2]) / r);
    double cs = sqrt(g.gamma * p / r);
    double ax = g.dx / (fabs(u) + cs);
    double ay = g.dy / (fabs(v) + cs);
    double a = ax < ay ? ax : ay;
    if (!(a > 0.0) || !isfinite(a)) bad = true;
    else best = a < best ? a : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    best = ob < best ? ob : best;
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&sc->err, kErrDt);
    if (best < INFINITY)
      atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(best));
  }
}

// fixed_dt > 0 takes that step; otherwise the CFL step, clipped to t_end
// when clip != 0
__global__ void k_dt_finalize(Scalars* sc, double cfl, double fixed_dt, int clip, double t_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double dt;
  if (fixed_dt > 0.0) {
    dt = fixed_dt;
  } else {
    dt = cfl * __longlong_as_double((long long)sc->dtmin_bits);
    if (clip && sc->t + dt > t_end) dt = t_end - sc->t;
  }
  if (!(dt > 0.0) || !isfinite(dt)) sc->err |= kErrDt;
  sc->dt = dt;
  sc->dtmin_bits = 0x7ff0000000000000ull;  // +inf for the next step
  for (int s = 0; s < 3; ++s) {
    sc->iters[s] = 0;
    sc->nbad_first[s] = 0;
    sc->nbad_total[s] = 0;
    sc->nfog_pad[s] = 0;
  }
  sc->count[0] = sc->count[1] = 0;
}

__global__ void k_finish_step(Scalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc->t += sc->dt;
  sc->nsteps += 1;
}


__global__ void k_mood_lower(MoodArgs M, uint8_t* ord, Cascade C) {
  const int n = *M.qcount;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int c = M.queue[q];
    ord[c] = (uint8_t)C.next[ord[c]];
    M.stamp[c] = M.cur;
  }
}


// bookkeeping after a pass that filled queue slot cur_slot
__global__ void k_mood_account(Scalars* sc, int stage, int cur_slot, int first) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = sc->count[cur_slot];
  if (first) sc->nbad_first[stage] = n;
  sc->nbad_total[stage] += n;
  if (!first) sc->iters[stage] += 1;
  sc->count[cur_slot ^ 1] = 0;
}


}  // namespace gpm
