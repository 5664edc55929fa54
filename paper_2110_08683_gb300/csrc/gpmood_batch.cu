// gpmood_batch.cu -- many independent GP-MOOD problems of uneven sizes
// advanced together (include/gpmood.h, gpmood_batch_*): pooled buffers, one
// persistent launch per kernel class walking (problem, block) work items,
// one captured graph per step with the MOOD loops as conditional WHILE
// nodes, per-problem time steps, and a small autotuner for the face kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/gpmood.h"
#include "gp_weights.h"
#include "gpmood_kernels.cuh"
#include "gpmood_launch.h"
#include "weight_tables.h"

using namespace gpm;

namespace gpm {

// per-problem time-step reduction over (problem, chunk) items
__global__ void k_dt_reduce_batch(const double* X, const float* Xf, const Prob* probs,
                                  Scalars* psc, Scalars* gsc, const Item* items, int nitems) {
  if (gsc->ctl.fixed_dt > 0.0) return;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const Item w = items[it];
    const Prob& P = probs[w.p];
    const Grid& g = P.g;
    const double* Xp = X + P.state_off;
    const float* Xfp = Xf ? Xf + P.state_off : nullptr;
    double best = 0.0;
    bool bad = false;
    const long long c0 = (long long)w.a * 4096;
    const long long c1 = c0 + 4096 < (long long)P.ncell ? c0 + 4096 : (long long)P.ncell;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      int i = (int)(c % g.nx), j = (int)(c / g.nx);
      double a;
      if (!cell_rate_at(Xp, Xfp, g, i, j, a)) bad = true;
      else best = a > best ? a : best;
    }
    if (w.a == 0 && threadIdx.x == 0 && g.rate_floor > best) best = g.rate_floor;
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = ob > best ? ob : best;
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
      if (bad) atomicOr(&gsc->err, kErrDt);
      if (best > 0.0)
        atomicMax(&psc[w.p].rate_bits, (unsigned long long)__double_as_longlong(best));
    }
  }
}

// per-problem step: given dt, or CFL clipped to t_end; a problem already at
// t_end gets dt = 0 and only carries its state over
__global__ void k_dt_finalize_batch(Scalars* psc, Scalars* gsc, int nprob) {
  const Control c = gsc->ctl;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    Scalars& s = psc[p];
    double dt;
    bool active = true;
    if (c.clip && !(s.t < c.t_end * (1.0 - 1e-14))) {
      dt = 0.0;
      active = false;
    } else if (c.fixed_dt > 0.0) {
      dt = c.fixed_dt;
    } else {
      dt = c.cfl / __longlong_as_double((long long)s.rate_bits);
      if (c.clip && s.t + dt > c.t_end) dt = c.t_end - s.t;
    }
    if (active && (!(dt > 0.0) || !isfinite(dt))) atomicOr(&gsc->err, kErrDt);
    s.dt = dt;
    s.rate_bits = 0ull;
    if (active) atomicAdd(&gsc->nactive, 1);
  }
}

__global__ void k_batch_reset(Scalars* gsc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int s = 0; s < 3; ++s) {
    gsc->iters[s] = 0;
    gsc->nbad_first[s] = 0;
    gsc->nbad_total[s] = 0;
    gsc->nfog_pad[s] = 0;
  }
  gsc->count[0] = gsc->count[1] = 0;
  gsc->nactive = 0;
}

__global__ void k_fill_batch(double* X, float* Xf, const Prob* probs, const Scalars* psc,
                             double tfrac, int nprob) {
  const int p = blockIdx.y;
  if (p >= nprob) return;
  const Prob& P = probs[p];
  const double t = psc[p].t + tfrac * psc[p].dt;
  const long long n = ghost_count(P.g);
  for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < n;
       tid += (long long)gridDim.x * blockDim.x)
    fill_ghost(X + P.state_off, Xf ? Xf + P.state_off : nullptr, P.g, t, tid);
}

__global__ void k_finish_batch(Scalars* psc, int nprob) {
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    psc[p].t += psc[p].dt;
    if (psc[p].dt > 0.0) psc[p].nsteps += 1;
  }
}

}  // namespace gpm

struct gpmood_batch_s {
  int nprob, top, precision, max_iters;
  Cascade cas;
  std::vector<Prob> hprobs;
  long long state_elems, fx_elems, fy_elems;
  int total_cells;
  cudaStream_t stream, cs, cs2;
  double* U[3];
  float* Uf[3];  // float shadows of U (FP32 path only, else null)
  void *Fx, *Fy;
  uint8_t *fb, *ord, *first;  // fb: face-state check bits, x faces then y faces
  uint32_t* stamp;     // two arrays of MOOD stamps over the pooled cells (odd, even values)
  int mood_blocks, coop;  // grid of the MOOD loop kernel; 1: cooperative launch
  int* queue[2];
  Prob* probs;
  Scalars *psc, *gsc;  // device: per problem and global
  Scalars* hgsc;       // pinned host mirror of the global scalars
  Item *items_fx[2], *items_fy[2], *items_up, *items_dt;  // [fw 4, fw 8]
  Item* items_xy;  // fused x+y face blocks: (problem, segment, band of 7 face rows)
  int n_fx[2], n_fy[2], n_up, n_dt, n_xy;
  ParityW<double> pw64;
  ParityW<float> pw32;
  DirectW<double> dw64;
  DirectW<float> dw32;
  Control ctl;
  int eager;  // stream launches instead of the captured step graph
  int cur, has_state;
  // face-kernel variant: fw[d] warps per block of sweep d (4 or 8), or
  // fw = {0, 0} for the fused x+y kernel; blocks: its work items
  int tuned, fw[2], blocks[2];
  int up_blocks, dt_blocks, fill_blocks_x;
  cudaGraphExec_t gexec[3][2];
  int prof_on;
  cudaEvent_t gev[64];
  int gev_cls[32], gev_n, gev_pairs;
  double prof_ms[GPMOOD_NKCLASS];
  long long prof_n[GPMOOD_NKCLASS];
};

namespace {

// CFL rate max((|u|+c)/dx, (|v|+c)/dy) of the jet inflow states of a grid's
// jet sides (0 without): those states enter the domain at the first step
double jet_rate(const Grid& g) {
  double r = 0.0;
  for (int side = 0; side < 2; ++side) {
    if (g.bc[2 + side] != 6) continue;
    const double* S = g.jetU[side];
    const double u = S[1] / S[0], v = S[2] / S[0];
    const double p = (g.gamma - 1.0) * (S[3] - 0.5 * (S[1] * u + S[2] * v));
    const double c = sqrt(g.gamma * p / S[0]);
    const double ax = (fabs(u) + c) / g.dx, ay = (fabs(v) + c) / g.dy;
    r = fmax(r, fmax(ax, ay));
  }
  return r;
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

void prim_to_cons(const double* P, double gam, double* U) {
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[0] * P[2];
  U[3] = P[3] / (gam - 1.0) + 0.5 * P[0] * (P[1] * P[1] + P[2] * P[2]);
}

#define CKB(call)                               \
  do {                                          \
    if ((call) != cudaSuccess) return GPMOOD_E_CUDA; \
  } while (0)

void batch_free(gpmood_batch_t b) {
  for (int k = 0; k < 64; ++k)
    if (b->gev[k]) cudaEventDestroy(b->gev[k]);
  for (int r = 0; r < 3; ++r)
    for (int p = 0; p < 2; ++p)
      if (b->gexec[r][p]) cudaGraphExecDestroy(b->gexec[r][p]);
  if (b->cs) cudaStreamDestroy(b->cs);
  if (b->cs2) cudaStreamDestroy(b->cs2);
  for (int k = 0; k < 3; ++k) {
    cudaFree(b->U[k]);
    cudaFree(b->Uf[k]);
  }
  void* ptrs[] = {b->Fx, b->Fy, b->fb, b->ord, b->first, b->stamp, b->queue[0], b->queue[1],
                  b->probs, b->psc, b->gsc, b->items_fx[0], b->items_fx[1], b->items_fy[0],
                  b->items_fy[1], b->items_up, b->items_dt, b->items_xy};
  for (void* p : ptrs) cudaFree(p);
  if (b->hgsc) cudaFreeHost(b->hgsc);
}

int upload_items(const std::vector<Item>& v, Item** out, int* n) {
  *n = (int)v.size();
  if (v.empty()) return 0;
  CKB(cudaMalloc(out, sizeof(Item) * v.size()));
  CKB(cudaMemcpy(*out, v.data(), sizeof(Item) * v.size(), cudaMemcpyHostToDevice));
  return 0;
}

template <class Real>
StageArgs<Real> batch_args(gpmood_batch_t b, int s, int ia, int ix, int io) {
  StageArgs<Real> A;
  // SSP-RK3 (eq. rk3): the stage combinations as out = ca U0 + cb Y
  static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
  A.h = 1.0;
  A.ca = ca[s];
  A.cb = cb[s];
  A.W = nullptr;
  A.out2 = nullptr;
  A.wa = A.wb = 0.0;
  A.X = b->U[ix];
  A.U0 = b->U[ia];
  A.out = b->U[io];
  if constexpr (sizeof(Real) == sizeof(float)) {
    A.Xr = b->Uf[ix];
    A.outr = b->Uf[io];
  } else {
    A.Xr = b->U[ix];
    A.outr = nullptr;
  }
  A.Fx = (double*)b->Fx;
  A.Fy = (double*)b->Fy;
  A.fbx = b->fb;
  A.fby = b->fb + b->fx_elems / 4;
  A.ord = b->ord + (size_t)s * b->total_cells;
  A.first = b->first + (size_t)s * b->total_cells;
  A.queue = b->queue[0];
  A.qcount = &b->gsc->count[0];
  A.sc = b->psc;
  A.scw = b->gsc;
  A.stage = s;
  return A;
}

int pull(gpmood_batch_t b) {
  CKB(cudaMemcpyAsync(b->hgsc, b->gsc, sizeof(Scalars), cudaMemcpyDeviceToHost, b->stream));
  CKB(cudaStreamSynchronize(b->stream));
  return 0;
}

int launch_dt_batch(gpmood_batch_t b, int ia, cudaStream_t st) {
  k_batch_reset<<<1, 32, 0, st>>>(b->gsc);
  k_dt_reduce_batch<<<b->dt_blocks, 256, 0, st>>>(b->U[ia], b->Uf[ia], b->probs, b->psc, b->gsc,
                                                  b->items_dt, b->n_dt);
  k_dt_finalize_batch<<<1, 256, 0, st>>>(b->psc, b->gsc, b->nprob);
  return cudaGetLastError() == cudaSuccess ? 0 : GPMOOD_E_CUDA;
}

int launch_fill_batch(gpmood_batch_t b, int ix, int s, cudaStream_t st) {
  static const double tfrac[3] = {0.0, 1.0, 0.5};
  k_fill_batch<<<dim3(b->fill_blocks_x, b->nprob), 256, 0, st>>>(b->U[ix], b->Uf[ix], b->probs,
                                                                  b->psc, tfrac[s], b->nprob);
  return cudaGetLastError() == cudaSuccess ? 0 : GPMOOD_E_CUDA;
}

template <class Real>
int launch_faces_batch(gpmood_batch_t b, int dir, const StageArgs<Real>& A,
                       const ParityW<Real>& P, int fw, int blocks, cudaStream_t st) {
  const int k = fw == 4 ? 0 : 1;
  Item* items = dir == 0 ? b->items_fx[k] : b->items_fy[k];
  int n = dir == 0 ? b->n_fx[k] : b->n_fy[k];
  return LaunchB<Real>::faces(b->top, dir, fw, A, b->probs, b->psc, items, n, blocks, P, st) ==
                 cudaSuccess
             ? 0
             : GPMOOD_E_CUDA;
}

// the first-pass faces of every problem in the tuned variant: the fused x+y
// kernel (fw = {0, 0}) or one sweep per direction
template <class Real>
int faces_b(gpmood_batch_t b, const StageArgs<Real>& A, const ParityW<Real>& P,
            cudaStream_t st) {
  if (b->fw[0] == 0)
    return LaunchB<Real>::faces_xy(b->top, A, b->probs, b->psc, b->items_xy, b->n_xy, P, st) ==
                   cudaSuccess
               ? 0
               : GPMOOD_E_CUDA;
  int rc = launch_faces_batch<Real>(b, 0, A, P, b->fw[0], b->blocks[0], st);
  if (!rc) rc = launch_faces_batch<Real>(b, 1, A, P, b->fw[1], b->blocks[1], st);
  return rc;
}

// the autotuner, on the first stage of the current state: the face kernels
// (per sweep 4 or 8 warps, i.e. rows, per work item; or the fused x+y
// kernel, one item per 31 x 7 faces of each direction) and the grid of the
// update kernel (blocks walking the update items); each variant is timed as
// the best of two runs after a warm-up run, and the fastest kept
template <class Real>
int tune(gpmood_batch_t b, const ParityW<Real>& P, const DirectW<Real>& D) {
  int rc = launch_dt_batch(b, b->cur, b->stream);
  if (rc) return rc;
  rc = launch_fill_batch(b, b->cur, 0, b->stream);
  if (rc) return rc;
  StageArgs<Real> A = batch_args<Real>(b, 0, b->cur, b->cur, (b->cur + 1) % 3);
  cudaEvent_t e0, e1;
  CKB(cudaEventCreate(&e0));
  CKB(cudaEventCreate(&e1));
  // best of runs 2 and 3 of launch(), ms; `before` runs untimed first
  auto timed = [&](auto launch, auto before) -> float {
    float ms_min = 1e30f;
    for (int rep = 0; rep < 3 && !rc; ++rep) {
      before();
      cudaEventRecord(e0, b->stream);
      rc = launch();
      cudaEventRecord(e1, b->stream);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;  // the first run warms up
    }
    return ms_min;
  };
  auto none = [] {};
  float split = 0.f;
  for (int dir = 0; dir < 2 && !rc; ++dir) {
    float best = 1e30f;
    for (int fw : {4, 8}) {
      const float ms =
          timed([&] { return launch_faces_batch<Real>(b, dir, A, P, fw, 0, b->stream); }, none);
      if (!rc && ms < best) {
        best = ms;
        b->fw[dir] = fw;
        b->blocks[dir] = dir == 0 ? b->n_fx[fw == 4 ? 0 : 1] : b->n_fy[fw == 4 ? 0 : 1];
      }
    }
    split += best;
  }
  const float fused = timed(
      [&] {
        return LaunchB<Real>::faces_xy(b->top, A, b->probs, b->psc, b->items_xy, b->n_xy, P,
                                       b->stream) == cudaSuccess
                   ? 0
                   : GPMOOD_E_CUDA;
      },
      none);
  if (!rc && fused < split) {
    b->fw[0] = b->fw[1] = 0;
    b->blocks[0] = b->blocks[1] = b->n_xy;
  }
  // the update kernel's grid; the queue and counters it fills are cleared
  // before every run
  float best_up = 1e30f;
  for (int k : {2, 4, 8, 16}) {
    const int nb = 152 * k < b->n_up ? 152 * k : b->n_up;
    const float ms = timed(
        [&] {
          return LaunchB<Real>::update(A, b->probs, b->psc, b->items_up, b->n_up, nb, D,
                                       b->stream) == cudaSuccess
                     ? 0
                     : GPMOOD_E_CUDA;
        },
        [&] { k_batch_reset<<<1, 32, 0, b->stream>>>(b->gsc); });
    if (!rc && ms < best_up) {
      best_up = ms;
      b->up_blocks = nb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->tuned = 1;
  return 0;
}

void rec(gpmood_batch_t b, int prof, int cls, int open, cudaStream_t st) {
  if (!prof) return;
  int k = b->gev_n;
  cudaEventRecordWithFlags(b->gev[k], st, cudaEventRecordExternal);
  if (!open) b->gev_cls[(k - 1) / 2] = cls;
  b->gev_n = k + 1;
}

// the MOOD loops of every problem in one launch; a driver that refuses the
// cooperative launch gets a plain launch of the same co-resident grid from
// then on (the kernel's barrier waits are bounded either way)
template <class Real>
int mood_loop_b(gpmood_batch_t b, const StageArgs<Real>& A, int s, const DirectW<Real>& D,
                cudaStream_t st) {
  MoodArgs M;
  M.queue[0] = b->queue[0];
  M.queue[1] = b->queue[1];
  M.stamp = b->stamp;
  M.stamp_stride = b->total_cells;
  M.sc = b->gsc;
  cudaError_t e = LaunchB<Real>::mood_loop(A, M, b->probs, b->psc, b->nprob, D, b->cas, s,
                                           b->mood_blocks, b->coop, st);
  if (e != cudaSuccess && b->coop) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      b->coop = 0;
      e = LaunchB<Real>::mood_loop(A, M, b->probs, b->psc, b->nprob, D, b->cas, s,
                                   b->mood_blocks, 0, st);
    }
  }
  CKB(e);
  return 0;
}

template <class Real>
int capture_stage_b(gpmood_batch_t b, int s, int ia, int ix, int io, const ParityW<Real>& P,
                    const DirectW<Real>& D, int prof) {
  cudaStream_t st = b->cs;
  StageArgs<Real> A = batch_args<Real>(b, s, ia, ix, io);
  rec(b, prof, GPMOOD_K_GHOST, 1, st);
  if (launch_fill_batch(b, ix, s, st)) return GPMOOD_E_CUDA;
  rec(b, prof, GPMOOD_K_GHOST, 0, st);
  rec(b, prof, GPMOOD_K_FACES_X, 1, st);
  if (faces_b<Real>(b, A, P, st)) return GPMOOD_E_CUDA;
  rec(b, prof, GPMOOD_K_FACES_X, 0, st);
  rec(b, prof, GPMOOD_K_FACES_Y, 1, st);
  rec(b, prof, GPMOOD_K_FACES_Y, 0, st);
  rec(b, prof, GPMOOD_K_UPDATE, 1, st);
  int nb = b->up_blocks < b->n_up ? b->up_blocks : b->n_up;
  CKB(LaunchB<Real>::update(A, b->probs, b->psc, b->items_up, b->n_up, nb, D, st));
  rec(b, prof, GPMOOD_K_UPDATE, 0, st);
  rec(b, prof, GPMOOD_K_MOOD, 1, st);
  int rc = mood_loop_b<Real>(b, A, s, D, st);
  if (rc) return rc;
  rec(b, prof, GPMOOD_K_MOOD, 0, st);
  return 0;
}

int capture_b(gpmood_batch_t b, int cur, int prof, cudaGraphExec_t* out) {
  const int a = cur, bb = (a + 1) % 3, c = (a + 2) % 3;
  const int in[3] = {a, bb, c}, outb[3] = {bb, c, bb};
  cudaStream_t st = b->cs;
  b->gev_n = 0;
  CKB(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = 0;
  rec(b, prof, GPMOOD_K_DT, 1, st);
  rc = launch_dt_batch(b, a, st);
  rec(b, prof, GPMOOD_K_DT, 0, st);
  for (int s = 0; s < 3 && !rc; ++s)
    rc = b->precision == GPMOOD_FP32
             ? capture_stage_b<float>(b, s, a, in[s], outb[s], b->pw32, b->dw32, prof)
             : capture_stage_b<double>(b, s, a, in[s], outb[s], b->pw64, b->dw64, prof);
  if (!rc) {
    k_finish_batch<<<1, 256, 0, st>>>(b->psc, b->nprob);
    if (cudaGetLastError() != cudaSuccess) rc = GPMOOD_E_CUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (!rc && ee != cudaSuccess) rc = GPMOOD_E_CUDA;
  if (!rc && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) rc = GPMOOD_E_CUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  if (!rc && prof) b->gev_pairs = b->gev_n / 2;
  return rc;
}

// the eager stage: the same kernels on the stream, the host reading the
// MOOD loop decision after every iteration
template <class Real>
int eager_stage_b(gpmood_batch_t b, int s, int ia, int ix, int io, const ParityW<Real>& P,
                  const DirectW<Real>& D) {
  cudaStream_t st = b->stream;
  StageArgs<Real> A = batch_args<Real>(b, s, ia, ix, io);
  if (launch_fill_batch(b, ix, s, st)) return GPMOOD_E_CUDA;
  if (faces_b<Real>(b, A, P, st)) return GPMOOD_E_CUDA;
  int nb = b->up_blocks < b->n_up ? b->up_blocks : b->n_up;
  CKB(LaunchB<Real>::update(A, b->probs, b->psc, b->items_up, b->n_up, nb, D, st));
  int rc = mood_loop_b<Real>(b, A, s, D, st);
  if (rc) return rc;
  return pull(b);
}

int eager_step_b(gpmood_batch_t b) {
  const int a = b->cur, bb = (a + 1) % 3, c = (a + 2) % 3;
  const int in[3] = {a, bb, c}, outb[3] = {bb, c, bb};
  int rc = launch_dt_batch(b, a, b->stream);
  for (int s = 0; s < 3 && !rc; ++s)
    rc = b->precision == GPMOOD_FP32
             ? eager_stage_b<float>(b, s, a, in[s], outb[s], b->pw32, b->dw32)
             : eager_stage_b<double>(b, s, a, in[s], outb[s], b->pw64, b->dw64);
  if (rc) return rc;
  k_finish_batch<<<1, 256, 0, b->stream>>>(b->psc, b->nprob);
  CKB(cudaGetLastError());
  return pull(b);
}

int batch_step(gpmood_batch_t b, double cfl, double fixed_dt, int clip, double t_end) {
  if (!b->has_state) return GPMOOD_E_NOSTATE;
  b->ctl.cfl = cfl;
  b->ctl.fixed_dt = fixed_dt;
  b->ctl.clip = clip;
  b->ctl.t_end = t_end;
  b->ctl.max_iters = b->max_iters;
  CKB(cudaMemcpyAsync(&b->gsc->ctl, &b->ctl, sizeof(Control), cudaMemcpyHostToDevice, b->stream));
  if (!b->tuned) {
    int rc = b->precision == GPMOOD_FP32 ? tune<float>(b, b->pw32, b->dw32)
                                         : tune<double>(b, b->pw64, b->dw64);
    if (rc) return rc;
  }
  const int prof = (b->prof_on && !b->eager) ? 1 : 0;
  if (b->eager) {
    int rc = eager_step_b(b);
    if (rc) return rc;
  } else {
    cudaGraphExec_t& ge = b->gexec[b->cur][prof];
    if (!ge) {
      int rc = capture_b(b, b->cur, prof, &ge);
      if (rc && b->coop) {
        // the CUDA driver refused a cooperative kernel node: a plain launch of
        // the same co-resident grid
        b->coop = 0;
        rc = capture_b(b, b->cur, prof, &ge);
      }
      if (rc) return rc;
    }
    CKB(cudaGraphLaunch(ge, b->stream));
    int rc = pull(b);
    if (rc) return rc;
  }
  if (prof) {
    for (int k = 0; k < b->gev_pairs; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b->gev[2 * k], b->gev[2 * k + 1]) == cudaSuccess)
        b->prof_ms[b->gev_cls[k]] += ms;
    }
    for (int k = GPMOOD_K_GHOST; k <= GPMOOD_K_FACES_Y; ++k) b->prof_n[k] += 3;
    b->prof_n[GPMOOD_K_DT] += 5;
    b->prof_n[GPMOOD_K_UPDATE] += 3;
    b->prof_n[GPMOOD_K_MOOD] += 3;
  }
  if (b->hgsc->err & kErrDt) return GPMOOD_E_DT;
  if (b->hgsc->err & kErrCap) return GPMOOD_E_MOOD_CAP;
  if (b->hgsc->err & kErrSync) return GPMOOD_E_SYNC;
  b->cur = (b->cur + 1) % 3;
  return GPMOOD_OK;
}

}  // namespace

extern "C" {

int gpmood_batch_create(const gpmood_grid* grids, int nprob, double gamma, int R_max,
                        const double* ell, const gpmood_options* opts, gpmood_batch_t* out) {
  if (!out) return GPMOOD_E_INVAL;
  *out = nullptr;
  if (!grids || !ell || nprob < 1 || R_max < 0 || R_max > 3 || !(gamma > 1.0))
    return GPMOOD_E_INVAL;
  gpmood_options o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  int cascade[4], nc = 0;
  if (o.ncascade == 0) {
    for (int r = R_max; r >= 0; --r) cascade[nc++] = r;
  } else {
    if (o.ncascade < 1 || o.ncascade > 4) return GPMOOD_E_INVAL;
    nc = o.ncascade;
    for (int k = 0; k < nc; ++k) cascade[k] = o.cascade[k];
    if (cascade[0] != R_max || cascade[nc - 1] != 0) return GPMOOD_E_INVAL;
    for (int k = 0; k + 1 < nc; ++k)
      if (!(cascade[k] > cascade[k + 1])) return GPMOOD_E_INVAL;
  }
  if (o.precision != GPMOOD_FP64 && o.precision != GPMOOD_FP32) return GPMOOD_E_INVAL;
  if (o.rk != 0 && o.rk != 3) return GPMOOD_E_INVAL;  // batches step with SSP-RK3
  if (o.riemann != 0 && o.riemann != 1) return GPMOOD_E_INVAL;
  if (o.recon != 0) return GPMOOD_E_INVAL;  // GP reconstruction only
  const int H = R_max + 1 > 2 ? R_max + 1 : 2;
  const int minn = H > 3 ? H : 3;
  // every problem shares the weights: the same ell/dx and ell/dy
  double lx0 = 0, ly0 = 0;
  for (int p = 0; p < nprob; ++p) {
    const gpmood_grid* gr = &grids[p];
    if (gr->nx < minn || gr->ny < minn || !(gr->x1 > gr->x0) || !(gr->y1 > gr->y0) ||
        !(ell[p] > 0.0) || (gr->dim != 0 && gr->dim != 2))
      return GPMOOD_E_INVAL;
    for (int s = 0; s < 4; ++s) {
      int k = gr->bc[s];
      if (k < 0 || k > 6 || (k == GPMOOD_BC_JET && s < 2) || (k == GPMOOD_BC_DMR_BOTTOM && s != 2) ||
          (k == GPMOOD_BC_DMR_TOP && s != 3))
        return GPMOOD_E_INVAL;
    }
    if ((gr->bc[0] == 0) != (gr->bc[1] == 0) || (gr->bc[2] == 0) != (gr->bc[3] == 0))
      return GPMOOD_E_INVAL;
    const double lx = ell[p] * gr->nx / (gr->x1 - gr->x0), ly = ell[p] * gr->ny / (gr->y1 - gr->y0);
    if (p == 0) {
      lx0 = lx;
      ly0 = ly;
    } else if (fabs(lx - lx0) > 1e-12 * lx0 || fabs(ly - ly0) > 1e-12 * ly0) {
      return GPMOOD_E_INVAL;
    }
  }
  gpmood_batch_t b = new (std::nothrow) gpmood_batch_s();
  if (!b) return GPMOOD_E_OOM;
  b->nprob = nprob;
  b->top = R_max;
  b->precision = o.precision;
  b->coop = 1;
  b->mood_blocks = b->precision == GPMOOD_FP32 ? LaunchB<float>::mood_loop_blocks()
                                               : LaunchB<double>::mood_loop_blocks();
  if (b->mood_blocks <= 0 ||
      (b->precision == GPMOOD_FP32 ? LaunchB<float>::prepare() : LaunchB<double>::prepare()) !=
          cudaSuccess) {
    cudaGetLastError();
    delete b;
    return GPMOOD_E_CUDA;
  }
  b->eager = o.eager ? 1 : 0;
  int widest = 0;
  for (int p = 0; p < nprob; ++p) {
    widest = grids[p].nx > widest ? grids[p].nx : widest;
    widest = grids[p].ny > widest ? grids[p].ny : widest;
  }
  b->max_iters = o.max_mood_iters > 0 ? o.max_mood_iters : 64 + 4 * widest;
  for (int r = 0; r < 4; ++r) b->cas.next[r] = b->cas.prev[r] = r;
  for (int k = 0; k + 1 < nc; ++k) {
    b->cas.next[cascade[k]] = cascade[k + 1];
    b->cas.prev[cascade[k + 1]] = cascade[k];
  }
  b->cas.top = R_max;
  // per-problem descriptors and pooled offsets
  b->hprobs.resize(nprob);
  long long soff = 0, fxo = 0, fyo = 0;
  int coff = 0;
  const size_t fsz = sizeof(double);  // face fluxes are FP64 on both paths
  std::vector<Item> fx4, fx8, fy4, fy8, up, dtl, xy;
  long long max_ghost = 0;
  for (int p = 0; p < nprob; ++p) {
    const gpmood_grid* gr = &grids[p];
    Prob& P = b->hprobs[p];
    memset(&P, 0, sizeof(P));
    Grid& g = P.g;
    g.nx = gr->nx;
    g.dim = 2;
    g.ny = gr->ny;
    g.H = H;
    g.pitch = round_up(g.nx + 2 * H, 32);
    g.gy = g.ny + 2 * H;
    g.vstride = (long long)g.pitch * g.gy;
    g.dx = (gr->x1 - gr->x0) / g.nx;
    g.dy = (gr->y1 - gr->y0) / g.ny;
    g.inv_dx = 1.0 / g.dx;
    g.inv_dy = 1.0 / g.dy;
    g.x0 = gr->x0;
    g.y0 = gr->y0;
    g.gamma = gamma;
    for (int s = 0; s < 4; ++s) {
      g.bc[s] = gr->bc[s];
      prim_to_cons(gr->bc_prim[s], gamma, g.bcU[s]);
    }
    g.periodic_x = gr->bc[0] == GPMOOD_BC_PERIODIC;
    g.periodic_y = gr->bc[2] == GPMOOD_BC_PERIODIC;
    prim_to_cons(gr->dmr_post, gamma, g.dmr_post);
    prim_to_cons(gr->dmr_pre, gamma, g.dmr_pre);
    g.dmr_wall_x0 = gr->dmr_wall_x0;
    g.dmr_xs0 = gr->dmr_xs0;
    g.dmr_xs_speed = gr->dmr_xs_speed;
    g.jet_x0 = gr->jet_x0;
    g.jet_x1 = gr->jet_x1;
    prim_to_cons(gr->jet_prim[0], gamma, g.jetU[0]);
    prim_to_cons(gr->jet_prim[1], gamma, g.jetU[1]);
    g.riemann = o.riemann;
    g.rate_floor = jet_rate(g);
    P.det.sigma_v = o.sigma_v > 0 ? o.sigma_v : 5.0;
    P.det.sigma_p = o.sigma_p > 0 ? o.sigma_p : 5.0;
    P.det.csd_on = o.csd_off ? 0 : 1;
    P.det.plateau_thr = fmin(g.dx * g.dx * g.dx, g.dy * g.dy * g.dy);
    P.det.delta = fmin(g.dx, g.dy);
    detect_derive(P.det, g);
    int da[25], db[25];
    double d2x[25], d2y[25];
    if (gpw_second_derivative(g.dx, g.dy, ell[p], da, db, d2x, d2y) != 5) {
      delete b;
      return GPMOOD_E_WEIGHTS;
    }
    for (int m = 0; m < 5; ++m) {
      P.d2x[m] = d2x[m];
      P.d2y[m] = d2y[m];
      P.d2xf[m] = (float)d2x[m];
      P.d2yf[m] = (float)d2y[m];
    }
    P.state_off = soff;
    P.fx_off = fxo;
    P.fy_off = fyo;
    P.cell_off = coff;
    P.ncell = g.nx * g.ny;
    soff += 4 * g.vstride;
    soff = (soff + 31) / 32 * 32;
    fxo += 4LL * g.ny * (g.nx + 1);
    fxo = (fxo + 31) / 32 * 32;
    fyo += 4LL * (g.ny + 1) * g.nx;
    fyo = (fyo + 31) / 32 * 32;
    coff += P.ncell;
    // work items
    for (int fw : {4, 8}) {
      auto& vx = fw == 4 ? fx4 : fx8;
      auto& vy = fw == 4 ? fy4 : fy8;
      const int sx = (g.nx + 1 + kSegFaces - 1) / kSegFaces, bx = (g.ny + fw - 1) / fw;
      for (int b2 = 0; b2 < bx; ++b2)
        for (int s2 = 0; s2 < sx; ++s2) vx.push_back(Item{p, s2, b2, 0});
      const int sy = (g.ny + 1 + kSegFaces - 1) / kSegFaces, by = (g.nx + fw - 1) / fw;
      for (int b2 = 0; b2 < by; ++b2)
        for (int s2 = 0; s2 < sy; ++s2) vy.push_back(Item{p, s2, b2, 0});
    }
    {
      const int sx = (g.nx + 1 + kSegFaces - 1) / kSegFaces, bb = (g.ny + 1 + kXYBand - 1) / kXYBand;
      for (int b2 = 0; b2 < bb; ++b2)
        for (int s2 = 0; s2 < sx; ++s2) xy.push_back(Item{p, s2, b2, 0});
    }
    for (int by = 0; by < (g.ny + 7) / 8; ++by)
      for (int bx = 0; bx < (g.nx + 31) / 32; ++bx) up.push_back(Item{p, bx, by, 0});
    for (int ch = 0; ch < (P.ncell + 4095) / 4096; ++ch) dtl.push_back(Item{p, ch, 0, 0});
    long long ngh = (long long)g.ny * 2 * H + 2LL * H * (g.nx + 2 * H);
    if (ngh > max_ghost) max_ghost = ngh;
  }
  b->state_elems = soff;
  b->fx_elems = fxo;
  b->fy_elems = fyo;
  b->total_cells = coff;
  b->fill_blocks_x = (int)((max_ghost + 255) / 256);
  if (b->fill_blocks_x > 64) b->fill_blocks_x = 64;
  // weights (shared): solve on the first grid
  {
    const Grid& g0 = b->hprobs[0].g;
    gpw_radius wr[4];
    memset(wr, 0, sizeof(wr));
    for (int k = 0; k < nc; ++k) {
      int R = cascade[k];
      if (R == 0) continue;
      if (gpw_solve(R, g0.dx, g0.dy, ell[0], &wr[R]) != 0) {
        delete b;
        return GPMOOD_E_WEIGHTS;
      }
    }
    const Prob& P0 = b->hprobs[0];
    fill_weights<double>(wr, R_max, P0.d2x, P0.d2y, b->pw64, b->dw64);
    fill_weights<float>(wr, R_max, P0.d2x, P0.d2y, b->pw32, b->dw32);
  }
  const size_t nc_all = (size_t)b->total_cells;
  bool ok = true;
  for (int k = 0; k < 3; ++k)
    ok = ok && cudaMalloc(&b->U[k], sizeof(double) * (size_t)b->state_elems) == cudaSuccess;
  if (b->precision == GPMOOD_FP32)
    for (int k = 0; k < 3; ++k)
      ok = ok && cudaMalloc(&b->Uf[k], sizeof(float) * (size_t)b->state_elems) == cudaSuccess;
  ok = ok && cudaMalloc(&b->Fx, fsz * (size_t)b->fx_elems) == cudaSuccess;
  ok = ok && cudaMalloc(&b->Fy, fsz * (size_t)b->fy_elems) == cudaSuccess;
  ok = ok && cudaMalloc(&b->fb, (size_t)(b->fx_elems + b->fy_elems) / 4) == cudaSuccess;
  ok = ok && cudaMalloc(&b->ord, 3 * nc_all) == cudaSuccess;
  ok = ok && cudaMalloc(&b->first, 3 * nc_all) == cudaSuccess;
  ok = ok && cudaMalloc(&b->stamp, 8 * nc_all) == cudaSuccess;
  ok = ok && cudaMalloc(&b->queue[0], 4 * nc_all) == cudaSuccess;
  ok = ok && cudaMalloc(&b->queue[1], 4 * nc_all) == cudaSuccess;
  ok = ok && cudaMalloc(&b->probs, sizeof(Prob) * nprob) == cudaSuccess;
  ok = ok && cudaMalloc(&b->psc, sizeof(Scalars) * nprob) == cudaSuccess;
  ok = ok && cudaMalloc(&b->gsc, sizeof(Scalars)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->hgsc, sizeof(Scalars)) == cudaSuccess;
  ok = ok && upload_items(fx4, &b->items_fx[0], &b->n_fx[0]) == 0;
  ok = ok && upload_items(fx8, &b->items_fx[1], &b->n_fx[1]) == 0;
  ok = ok && upload_items(fy4, &b->items_fy[0], &b->n_fy[0]) == 0;
  ok = ok && upload_items(fy8, &b->items_fy[1], &b->n_fy[1]) == 0;
  ok = ok && upload_items(up, &b->items_up, &b->n_up) == 0;
  ok = ok && upload_items(dtl, &b->items_dt, &b->n_dt) == 0;
  ok = ok && upload_items(xy, &b->items_xy, &b->n_xy) == 0;
  ok = ok && cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->cs2, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 64 && ok; ++k) ok = cudaEventCreate(&b->gev[k]) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(b->probs, b->hprobs.data(), sizeof(Prob) * nprob, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemset(b->fb, 0, (size_t)(b->fx_elems + b->fy_elems) / 4) == cudaSuccess &&
         cudaMemset(b->ord, 0, 3 * nc_all) == cudaSuccess &&
         cudaMemset(b->first, 0, 3 * nc_all) == cudaSuccess &&
         cudaMemset(b->stamp, 0, 8 * nc_all) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  for (int k = 0; k < 3 && ok; ++k)
    ok = cudaMemset(b->U[k], 0, sizeof(double) * (size_t)b->state_elems) == cudaSuccess &&
         (!b->Uf[k] ||
          cudaMemset(b->Uf[k], 0, sizeof(float) * (size_t)b->state_elems) == cudaSuccess);
  if (!ok) {
    batch_free(b);
    delete b;
    cudaGetLastError();
    return GPMOOD_E_OOM;
  }
  b->up_blocks = 152 * 8;
  b->dt_blocks = b->n_dt < 152 * 4 ? b->n_dt : 152 * 4;
  b->fw[0] = b->fw[1] = 8;
  b->blocks[0] = b->blocks[1] = 152 * 2;
  b->stream = nullptr;
  *out = b;
  return GPMOOD_OK;
}

int gpmood_batch_set_stream(gpmood_batch_t b, void* stream) {
  if (!b) return GPMOOD_E_INVAL;
  b->stream = (cudaStream_t)stream;
  return GPMOOD_OK;
}

int gpmood_batch_set_state(gpmood_batch_t b, const double* U, int on_device) {
  if (!b || !U) return GPMOOD_E_INVAL;
  b->cur = 0;
  size_t off = 0;
  for (int p = 0; p < b->nprob; ++p) {
    const Prob& P = b->hprobs[p];
    const Grid& g = P.g;
    for (int v = 0; v < 4; ++v) {
      double* dst = b->U[0] + P.state_off + v * g.vstride + (size_t)g.H * g.pitch + g.H;
      CKB(cudaMemcpy2DAsync(dst, sizeof(double) * g.pitch, U + off, sizeof(double) * g.nx,
                            sizeof(double) * g.nx, g.ny,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            b->stream));
      off += (size_t)g.nx * g.ny;
    }
  }
  if (b->Uf[0]) {
    k_to_real<float><<<152 * 8, 256, 0, b->stream>>>(b->U[0], b->Uf[0], b->state_elems);
    CKB(cudaGetLastError());
  }
  std::vector<Scalars> z(b->nprob);
  for (auto& s : z) {
    memset(&s, 0, sizeof(s));
    s.rate_bits = 0ull;
  }
  CKB(cudaMemcpyAsync(b->psc, z.data(), sizeof(Scalars) * b->nprob, cudaMemcpyHostToDevice,
                      b->stream));
  CKB(cudaMemcpyAsync(b->gsc, z.data(), sizeof(Scalars), cudaMemcpyHostToDevice, b->stream));
  CKB(cudaMemsetAsync(b->stamp, 0, 8 * (size_t)b->total_cells, b->stream));
  CKB(cudaStreamSynchronize(b->stream));
  b->has_state = 1;
  return GPMOOD_OK;
}

int gpmood_batch_get_state(gpmood_batch_t b, double* U, int on_device) {
  if (!b || !U) return GPMOOD_E_INVAL;
  if (!b->has_state) return GPMOOD_E_NOSTATE;
  size_t off = 0;
  for (int p = 0; p < b->nprob; ++p) {
    const Prob& P = b->hprobs[p];
    const Grid& g = P.g;
    for (int v = 0; v < 4; ++v) {
      const double* src = b->U[b->cur] + P.state_off + v * g.vstride + (size_t)g.H * g.pitch + g.H;
      CKB(cudaMemcpy2DAsync(U + off, sizeof(double) * g.nx, src, sizeof(double) * g.pitch,
                            sizeof(double) * g.nx, g.ny,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            b->stream));
      off += (size_t)g.nx * g.ny;
    }
  }
  CKB(cudaStreamSynchronize(b->stream));
  return GPMOOD_OK;
}

int gpmood_batch_step(gpmood_batch_t b, double cfl) {
  if (!b || !(cfl > 0.0)) return GPMOOD_E_INVAL;
  return batch_step(b, cfl, 0.0, 0, 0.0);
}

int gpmood_batch_run(gpmood_batch_t b, double t_end, double cfl, long long* nsteps_out) {
  if (!b || !(cfl > 0.0)) return GPMOOD_E_INVAL;
  long long n = 0;
  for (;;) {
    int rc = batch_step(b, cfl, 0.0, 1, t_end);
    if (rc) return rc;
    if (b->hgsc->nactive == 0) break;
    ++n;
  }
  if (nsteps_out) *nsteps_out = n;
  return GPMOOD_OK;
}

int gpmood_batch_info(gpmood_batch_t b, double* t, double* dt, long long* nsteps,
                      gpmood_stats* total) {
  if (!b) return GPMOOD_E_INVAL;
  std::vector<Scalars> s(b->nprob);
  CKB(cudaMemcpyAsync(s.data(), b->psc, sizeof(Scalars) * b->nprob, cudaMemcpyDeviceToHost,
                      b->stream));
  int rc = pull(b);
  if (rc) return rc;
  for (int p = 0; p < b->nprob; ++p) {
    if (t) t[p] = s[p].t;
    if (dt) dt[p] = s[p].dt;
    if (nsteps) nsteps[p] = s[p].nsteps;
  }
  if (total) {
    memset(total, 0, sizeof(*total));
    const Scalars& g = *b->hgsc;
    for (int k = 0; k < 3; ++k) {
      total->iters[k] = g.iters[k];
      total->nbad_first[k] = g.nbad_first[k];
      total->nbad_total[k] = g.nbad_total[k];
      total->nfog_pad[k] = g.nfog_pad[k];
    }
    total->status = GPMOOD_OK;
  }
  return GPMOOD_OK;
}

int gpmood_batch_tuning(gpmood_batch_t b, int* warps, int* blocks) {
  if (!b) return GPMOOD_E_INVAL;
  for (int d = 0; d < 2; ++d) {
    if (warps) warps[d] = b->fw[d];
    if (blocks) blocks[d] = b->blocks[d];
  }
  return b->tuned ? GPMOOD_OK : GPMOOD_E_NOSTATE;
}

int gpmood_batch_grids(gpmood_batch_t b, int* update_blocks, int* mood_blocks) {
  if (!b) return GPMOOD_E_INVAL;
  if (update_blocks) *update_blocks = b->up_blocks;
  if (mood_blocks) *mood_blocks = b->mood_blocks;
  return b->tuned ? GPMOOD_OK : GPMOOD_E_NOSTATE;
}

int gpmood_batch_profile(gpmood_batch_t b, int enable) {
  if (!b) return GPMOOD_E_INVAL;
  CKB(cudaStreamSynchronize(b->stream));
  b->prof_on = enable ? 1 : 0;
  if (enable)
    for (int k = 0; k < GPMOOD_NKCLASS; ++k) {
      b->prof_ms[k] = 0.0;
      b->prof_n[k] = 0;
    }
  return GPMOOD_OK;
}

int gpmood_batch_kernel_times(gpmood_batch_t b, double* ms, long long* launches) {
  if (!b) return GPMOOD_E_INVAL;
  CKB(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < GPMOOD_NKCLASS; ++k) {
    if (ms) ms[k] = b->prof_ms[k];
    if (launches) launches[k] = b->prof_n[k];
  }
  return GPMOOD_OK;
}

int gpmood_batch_destroy(gpmood_batch_t b) {
  if (!b) return GPMOOD_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  return GPMOOD_OK;
}

}  // extern "C"
