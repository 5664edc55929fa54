// common_kernels.cuh -- precision-independent kernels (ghost fill, time step,
// MOOD bookkeeping); included by the host driver only.
#pragma once

#include "gpmood_kernels.cuh"

namespace gpm {

__global__ void k_fill_ghosts(double* X, float* Xf, Grid g, const Scalars* sc, double tfrac) {
  pdl_wait();
  pdl_trigger();
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  fill_ghost(X, Xf, g, sc->t + tfrac * sc->dt, tid);
}

// time step: min over cells of min(dx/(|u|+c), dy/(|v|+c)), per-direction
// CFL form; positive doubles order like their bit patterns
// Xf: the float shadow of X on the FP32 path (the rate in float), else null
__global__ void k_dt_reduce(const double* X, const float* Xf, Grid g, Scalars* sc) {
  pdl_wait();
  pdl_trigger();
  if (sc->ctl.fixed_dt > 0.0) return;
  if (sc->rate_ready) {
    // the previous step's last MOOD loop kernel reduced the rate already
    if (blockIdx.x == 0 && threadIdx.x == 0 && sc->rate_bad) atomicOr(&sc->err, kErrDt);
    return;
  }
  double best = 0.0;
  bool bad = false;
  const long long n = (long long)g.nx * g.ny;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx), j = (int)(c / g.nx);
    double a;
    if (!cell_rate_at(X, Xf, g, i, j, a)) bad = true;
    else best = a > best ? a : best;
  }
  // the inflow state of a jet boundary enters at the first step: its rate counts
  if (blockIdx.x == 0 && threadIdx.x == 0 && g.rate_floor > best) best = g.rate_floor;
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    best = ob > best ? ob : best;
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&sc->err, kErrDt);
    // positive doubles order as their bit patterns
    if (best > 0.0) atomicMax(&sc->rate_bits, (unsigned long long)__double_as_longlong(best));
  }
}

// the step: a given dt (ctl.fixed_dt > 0) or the CFL step, clipped to
// ctl.t_end when ctl.clip != 0; zeroes the per-step counters
__global__ void k_dt_finalize(Scalars* sc) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Control c = sc->ctl;
  double dt;
  if (c.fixed_dt > 0.0) {
    dt = c.fixed_dt;
  } else {
    dt = c.cfl / __longlong_as_double((long long)sc->rate_bits);
    if (c.clip && sc->t + dt > c.t_end) dt = c.t_end - sc->t;
  }
  if (!(dt > 0.0) || !isfinite(dt)) sc->err |= kErrDt;
  sc->dt = dt;
  sc->rate_bits = 0ull;  // +0 for the next step
  sc->rate_ready = 0;
  sc->rate_bad = 0;
  for (int s = 0; s < 5; ++s) {
    sc->iters[s] = 0;
    sc->nbad_first[s] = 0;
    sc->nbad_total[s] = 0;
    sc->nfog_pad[s] = 0;
  }
  sc->count[0] = sc->count[1] = 0;
}

// end of a step: a failed step (non-finite dt, MOOD cap) leaves the time and
// the step count where they were.  `base` is the step's launch count, added
// to the running count.
__global__ void k_finish_step(Scalars* sc, int base) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (sc->err == 0) {
    sc->t += sc->dt;
    sc->nsteps += 1;
  }
  sc->launches += base;
}

// gate of an asynchronous graph step: the step runs while no error is latched
// and, for a clipped run, while t < t_end (the host's own loop test).  Once
// closed the gate stays closed for the following steps, so the steps that ran
// are always a prefix of those launched.
__global__ void k_step_gate(Scalars* sc, cudaGraphConditionalHandle hif) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Control c = sc->ctl;
  bool go = sc->err == 0;
  if (c.clip && !(sc->t < c.t_end * (1.0 - 1e-14))) go = false;
  if (!go) sc->launches += 1;  // the gate alone
  cudaGraphSetConditional(hif, go ? 1u : 0u);
}


// ---------------------------------------------------------------------------
// adjoint helpers
// ---------------------------------------------------------------------------
__global__ void k_fill_ghosts_at(double* X, Grid g, double t) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  fill_ghost(X, nullptr, g, t, tid);
}

// transpose of the ghost fill: every ghost cell's adjoint goes to the
// cell it was copied from, the y rule first (all columns, corners included)
// and then the x rule (interior rows), the reverse of the fill's
// composition; fixed states drop out.  One thread walks the ghosts of one
// line in a fixed order, so the sums do not depend on scheduling.

// source row and sign of the normal momentum of y ghost row j in column i;
// false: a fixed state
__device__ __forceinline__ bool fold_src_y(const Grid& g, int i, int j, int& sj, double& sgn) {
  const int side = j < 0 ? 0 : 1;
  const int k = j < 0 ? -j : j - g.ny + 1;
  const int kind = g.bc[2 + side];
  bool reflect = kind == 2;
  if (kind == 3 || kind == 5) return false;
  if (kind == 6) {  // jet: fixed inside the slit, outflow elsewhere
    const double xc = g.x0 + (i + 0.5) * g.dx;
    if (xc >= g.jet_x0 && xc <= g.jet_x1) return false;
  }
  if (kind == 4) {
    const double xc = g.x0 + (i + 0.5) * g.dx;
    if (xc < g.dmr_wall_x0) return false;
    reflect = true;
  }
  if (kind == 0) sj = wrapi(j, g.ny);
  else if (reflect) sj = side == 0 ? k - 1 : g.ny - k;
  else sj = side == 0 ? 0 : g.ny - 1;
  sgn = reflect ? -1.0 : 1.0;
  return true;
}

__device__ __forceinline__ bool fold_src_x(const Grid& g, int i, int& si, double& sgn) {
  const int side = i < 0 ? 0 : 1;
  const int k = i < 0 ? -i : i - g.nx + 1;
  const int kind = g.bc[side];
  if (kind == 3) return false;
  if (kind == 0) si = wrapi(i, g.nx);
  else if (kind == 2) si = side == 0 ? k - 1 : g.nx - k;
  else si = side == 0 ? 0 : g.nx - 1;
  sgn = kind == 2 ? -1.0 : 1.0;
  return true;
}

// one thread per ghosted column i in [-H, nx+H)
__global__ void k_adj_fold_y(double* G, Grid g) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - g.H;
  if (i >= g.nx + g.H) return;
  for (int side = 0; side < 2; ++side)
    for (int k = 1; k <= g.H; ++k) {
      const int j = side == 0 ? -k : g.ny - 1 + k;
      int sj;
      double sgn;
      if (!fold_src_y(g, i, j, sj, sgn)) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v)
        G[gidx(g, v, i, sj)] += (v == 2 ? sgn : 1.0) * G[gidx(g, v, i, j)];
    }
}

// one thread per interior row j
__global__ void k_adj_fold_x(double* G, Grid g) {
  const int j = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= g.ny) return;
  for (int side = 0; side < 2; ++side)
    for (int k = 1; k <= g.H; ++k) {
      const int i = side == 0 ? -k : g.nx - 1 + k;
      int si;
      double sgn;
      if (!fold_src_x(g, i, si, sgn)) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v)
        G[gidx(g, v, si, j)] += (v == 1 ? sgn : 1.0) * G[gidx(g, v, i, j)];
    }
}

// w = v - dt G (interior of the ghosted G)
__global__ void k_adj_stage_out(double* w, const double* v, const double* G, Grid g, double dt) {
  const long long nc = (long long)g.nx * g.ny;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < 4 * nc;
       t += (long long)gridDim.x * blockDim.x) {
    const int vv = (int)(t / nc);
    const long long c = t - vv * nc;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    w[t] = v[t] - dt * G[gidx(g, vv, i, j)];
  }
}

// tape of a recorded step: the interior of stage input s, and the radii
// of stage s, into the destinations the step's controls name
__global__ void k_tape_state(const double* X, Grid g, const Scalars* sc, int s) {
  double* dst = sc->ctl.tape;
  if (!dst) return;
  const long long nc = (long long)g.nx * g.ny;
  dst += (long long)s * 4 * nc;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < 4 * nc;
       t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / nc);
    const long long c = t - v * nc;
    dst[t] = X[gidx(g, v, (int)(c % g.nx), (int)(c / g.nx))];
  }
}

__global__ void k_tape_ord(const uint8_t* ord, const Scalars* sc, int s, long long nc) {
  uint8_t* dst = sc->ctl.otape;
  if (!dst) return;
  dst += s * nc;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = ord[t];
}

// out = a x + b y (b = 0: y unused)
__global__ void k_lincomb(double* out, double a, const double* x, double b, const double* y,
                          long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = b == 0.0 ? a * x[t] : a * x[t] + b * y[t];
}

// interior cell averages [4][ny][nx] (src: device memory or pinned host
// memory read over the chip-to-chip link) into a ghosted state X and, on the
// FP32 path, its float shadow Xf: one pass, coalesced on both sides
__global__ void k_set_interior(const double* __restrict__ src, double* X, float* Xf, Grid g) {
  const long long n = 4LL * g.nx * g.ny;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / ((long long)g.nx * g.ny));
    const long long r = t - (long long)v * g.nx * g.ny;
    const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
    const long long k = v * g.vstride + (long long)(j + g.H) * g.pitch + (i + g.H);
    const double x = src[t];
    X[k] = x;
    if (Xf) Xf[k] = (float)x;
  }
}

// the interior of a ghosted state X out to [4][ny][nx] (device memory or
// pinned host memory written over the chip-to-chip link)
__global__ void k_get_interior(const double* X, double* __restrict__ dst, Grid g) {
  const long long n = 4LL * g.nx * g.ny;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / ((long long)g.nx * g.ny));
    const long long r = t - (long long)v * g.nx * g.ny;
    const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
    dst[t] = X[v * g.vstride + (long long)(j + g.H) * g.pitch + (i + g.H)];
  }
}

}  // namespace gpm
