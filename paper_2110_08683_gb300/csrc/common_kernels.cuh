// common_kernels.cuh -- precision-independent kernels (ghost fill, time step,
// MOOD bookkeeping); included by the host driver only.
#pragma once

#include "gpmood_kernels.cuh"

namespace gpm {

__global__ void k_fill_ghosts(double* X, Grid g, const Scalars* sc, double tfrac) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  fill_ghost(X, g, sc->t + tfrac * sc->dt, tid);
}

// time step: min over cells of min(dx/(|u|+c), dy/(|v|+c)), per-direction
// CFL form; positive doubles order like their bit patterns
__global__ void k_dt_reduce(const double* X, Grid g, Scalars* sc) {
  if (sc->ctl.fixed_dt > 0.0) return;
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

// the step: a given dt (ctl.fixed_dt > 0) or the CFL step, clipped to
// ctl.t_end when ctl.clip != 0; zeroes the per-step counters
__global__ void k_dt_finalize(Scalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Control c = sc->ctl;
  double dt;
  if (c.fixed_dt > 0.0) {
    dt = c.fixed_dt;
  } else {
    dt = c.cfl * __longlong_as_double((long long)sc->dtmin_bits);
    if (c.clip && sc->t + dt > c.t_end) dt = c.t_end - sc->t;
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
  const int slot = M.sc->slot;
  const int n = M.sc->count[slot];
  const int* queue = M.queue[slot];
  const uint32_t cur = M.sc->stamp_cur;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int c = queue[q];
    ord[c] = (uint8_t)C.next[ord[c]];
    M.stamp[c] = cur;
  }
}

// decide whether another MOOD iteration runs; mirrors it into sc->go and,
// inside a captured graph, into the WHILE node's condition
__device__ __forceinline__ void mood_decide(Scalars* sc, int stage, int n,
                                            cudaGraphConditionalHandle hc, int use_graph) {
  int go = n > 0;
  if (go && sc->iters[stage] >= sc->ctl.max_iters) {
    sc->err |= kErrCap;
    go = 0;
  }
  if (go) sc->stamp_cur += 1;  // fresh stamp for the queue about to be worked on
  sc->go = go;
  if (use_graph) cudaGraphSetConditional(hc, go ? 1u : 0u);
}

// after the first pass (which filled queue 0)
__global__ void k_mood_begin(Scalars* sc, int stage, cudaGraphConditionalHandle hc, int use_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = sc->count[0];
  sc->slot = 0;
  sc->count[1] = 0;
  sc->nbad_first[stage] = n;
  sc->nbad_total[stage] = n;
  sc->iters[stage] = 0;
  mood_decide(sc, stage, n, hc, use_graph);
}

// after one MOOD iteration (which filled the other queue)
__global__ void k_mood_end(Scalars* sc, int stage, cudaGraphConditionalHandle hc, int use_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int s = sc->slot, ns = s ^ 1;
  const int n = sc->count[ns];
  sc->nbad_total[stage] += n;
  sc->iters[stage] += 1;
  sc->count[s] = 0;
  sc->slot = ns;
  mood_decide(sc, stage, n, hc, use_graph);
}

}  // namespace gpm
