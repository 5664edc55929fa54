// gpmood_api.cu -- the C ABI (include/gpmood.h): handle, buffers, weights,
// and the host driver of one SSP-RK3 step with the MOOD loop per stage.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "../../include/gpmood.h"
#include "common_kernels.cuh"
#include "gp_weights.h"
#include "gpmood_launch.h"
#include "weight_tables.h"

using namespace gpm;
using gpm::fill_weights;

struct gpmood_s {
  Grid g;
  Cascade cas;
  Detect det;
  int precision;
  int max_iters;
  cudaStream_t stream;
  Scheme sch;      // the RK scheme as stage roles and coefficients
  double* U[5];    // state buffers (3 for SSP-RK3, 5 for SSP-RK4)
  float* Uf[5];    // float shadows of U (FP32 path only, else null)
  void* Fx;
  void* Fy;
  uint8_t* fb;     // face-state check bits: x faces, then y faces
  uint8_t* ord;    // [S][nc], S stages
  uint8_t* first;  // [S][nc]
  uint32_t* stamp;  // two arrays of ncell MOOD stamps (odd and even values)
  int* queue[2];
  Scalars* sc;     // device
  Scalars* hsc;    // pinned host mirror
  ParityW<double> pw64;
  ParityW<float> pw32;
  DirectW<double> dw64;
  DirectW<float> dw32;
  int cur;         // buffer holding U^n
  int has_state;
  int launches;
  int last_status;
  int mood_blocks;  // grid of the MOOD loop kernel (co-resident blocks)
  int split_faces;  // 1: one first-pass face kernel per direction
  int coop;         // 1: the MOOD loop kernel is launched cooperatively
  // optional per-class event timing (graph steps)
  int prof_on;
  double prof_ms[GPMOOD_NKCLASS];
  long long prof_n[GPMOOD_NKCLASS];
  // captured step graphs [buffer rotation][profiled] and their streams
  Control ctl;  // host copy of the step controls
  int eager;    // stream launches instead of the captured step graph
  cudaStream_t cs, cs2, cs3;   // capture streams: step, MOOD loop body, gated step body
  cudaGraphExec_t gexec[5][3];  // [rotation][plain, profiled, recording]
  // asynchronous steps: plain step graphs open with a gate (an IF node), so
  // steps can be queued without reading anything back; the host settles its
  // buffer rotation from the device's step count when it next synchronises
  int gated_ok;              // 0 not yet known, 1 plain graphs gated, -1 gating unavailable
  int pdl;                   // 1: programmatic dependent launch between step kernels
  int pend;                  // steps queued since the last settle
  int sync_cur;              // rotation at the last settle
  long long sync_nsteps;     // device step count at the last settle
  Control ctl_dev;           // controls last copied to the device
  int ctl_valid;
  cudaEvent_t gev[64];
  int gev_cls[32];
  int gev_n, gev_pairs;
  // adjoint work buffers (allocated on first use)
  double* aX;     // ghosted stage input
  void* aXr;      // its float copy (FP32 adjoint)
  double* aG;     // ghosted state adjoint
  double *av, *aw, *amu;  // interior vectors
  AdjFaces ax, ay;
  uint8_t* aord;
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

// a pointer kernels may dereference: device memory as given (on_device), or
// page-locked host memory through its device mapping; null for pageable
// host memory, which goes through the CUDA driver's staged copies
const double* device_view(const double* p, int on_device) {
  if (on_device) return p;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return (const double*)a.devicePointer;
  return nullptr;
}

int set_err(gpmood_t h, int code) {
  if (h) h->last_status = code;
  return code;
}

#define CK(call)                                \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return set_err(h, GPMOOD_E_CUDA); \
  } while (0)

void free_all(gpmood_t h) {
  for (int k = 0; k < 64; ++k)
    if (h->gev[k]) cudaEventDestroy(h->gev[k]);
  for (int r = 0; r < 5; ++r)
    for (int p = 0; p < 3; ++p)
      if (h->gexec[r][p]) cudaGraphExecDestroy(h->gexec[r][p]);
  if (h->cs) cudaStreamDestroy(h->cs);
  if (h->cs2) cudaStreamDestroy(h->cs2);
  if (h->cs3) cudaStreamDestroy(h->cs3);
  void* adj[] = {h->aX, h->aXr, h->aG, h->av, h->aw, h->amu, h->ax.L, h->ax.R, h->ax.K,
                 h->ay.L, h->ay.R, h->ay.K, h->aord};
  for (void* p : adj) cudaFree(p);
  for (int k = 0; k < 5; ++k) {
    cudaFree(h->U[k]);
    cudaFree(h->Uf[k]);
  }
  cudaFree(h->Fx);
  cudaFree(h->Fy);
  cudaFree(h->fb);
  cudaFree(h->ord);
  cudaFree(h->first);
  cudaFree(h->stamp);
  cudaFree(h->queue[0]);
  cudaFree(h->queue[1]);
  cudaFree(h->sc);
  if (h->hsc) cudaFreeHost(h->hsc);
}

// the time integrators as stage roles.  SSP-RK3 (eq. rk3): three buffers
// rotating by one per step.  SSP-RK4 (eq. rk4, five stages), each stage
//   U^(s+1) = a_s U^n + b_s U^(s) - g_s Dt F(U^(s)) = a_s U^n + b_s Y_s,
// Y_s = U^(s) - (g_s / b_s) Dt F(U^(s)) its forward-Euler sub-step (the MOOD
// candidate), and U^{n+1} = e2 U^(2) + e3 Y_3 + e4 Y_4 with
// Y_4 = U^(4) - (f4 / e4) Dt F(U^(4)); e3 Y_3 = e3 U^(3) - f3 Dt F(U^(3)) (the
// printed plus sign of that term read as a minus).  Buffers: 0 U^n, 1 U^(1)
// then U^(4), 2 U^(2), 3 U^(3), 4 e2 U^(2) + e3 Y_3; the last stage writes
// U^{n+1} over U^n, so the buffers do not rotate.
void make_scheme(int rk, Scheme* S) {
  memset(S, 0, sizeof(*S));
  if (rk != 4) {
    S->nstages = 3;
    S->nbuf = 3;
    S->advance = 1;
    S->st[0] = {0, 1, 0, -1, -1, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0};
    S->st[1] = {1, 2, 0, -1, -1, 1.0, 0.75, 0.25, 0.0, 0.0, 1.0};
    S->st[2] = {2, 1, 0, -1, -1, 1.0, 1.0 / 3.0, 2.0 / 3.0, 0.0, 0.0, 0.5};
    return;
  }
  const double a[4] = {0.0, 0.444370493651235, 0.620101851488403, 0.178079954393132};
  const double b[4] = {1.0, 0.555629506348765, 0.379898148511597, 0.821920045606868};
  const double g[4] = {0.391752226571890, 0.368410593050371, 0.251891774271694,
                       0.544974750228521};
  const double e2 = 0.517231671970585, e3 = 0.096059710526147, e4 = 0.386708617503269;
  const double f4 = 0.226007483236906;
  S->nstages = 5;
  S->nbuf = 5;
  S->advance = 0;
  double c = 0.0;  // time of U^(s) over Dt
  const int in[4] = {0, 1, 2, 3}, out[4] = {1, 2, 3, 1};
  for (int s = 0; s < 4; ++s) {
    S->st[s] = {in[s], out[s], 0, -1, -1, g[s] / b[s], a[s], b[s], 0.0, 0.0, c};
    c = b[s] * c + g[s];
  }
  S->st[3].w = 2;
  S->st[3].out2 = 4;
  S->st[3].wa = e2;
  S->st[3].wb = e3;
  S->st[4] = {1, 0, 4, -1, -1, f4 / e4, 1.0, e4, 0.0, 0.0, c};
}

// buffer holding slot `slot` of the scheme in rotation `rot`
int buf_of(gpmood_t h, int rot, int slot) { return (rot + slot) % h->sch.nbuf; }

template <class Real>
StageArgs<Real> stage_args(gpmood_t h, int s, int rot) {
  StageArgs<Real> A;
  const StageSpec& p = h->sch.st[s];
  const int ix = buf_of(h, rot, p.in), io = buf_of(h, rot, p.out), ia = buf_of(h, rot, p.u0);
  const size_t nc = (size_t)h->g.nx * h->g.ny;
  A.h = p.h;
  A.ca = p.ca;
  A.cb = p.cb;
  A.W = p.w >= 0 ? h->U[buf_of(h, rot, p.w)] : nullptr;
  A.out2 = p.out2 >= 0 ? h->U[buf_of(h, rot, p.out2)] : nullptr;
  A.wa = p.wa;
  A.wb = p.wb;
  A.X = h->U[ix];
  A.U0 = h->U[ia];
  A.out = h->U[io];
  if constexpr (sizeof(Real) == sizeof(float)) {
    A.Xr = h->Uf[ix];
    A.outr = h->Uf[io];
  } else {
    A.Xr = h->U[ix];
    A.outr = nullptr;
  }
  A.Fx = (double*)h->Fx;
  A.Fy = (double*)h->Fy;
  A.fbx = h->fb;
  A.fby = h->fb + (size_t)(h->g.nx + 1) * h->g.ny;
  A.ord = h->ord + s * nc;
  A.first = h->first + s * nc;
  A.queue = h->queue[0];
  A.qcount = &h->sc->count[0];  // the first pass fills queue 0
  A.sc = h->sc;
  A.scw = h->sc;
  A.stage = s;
  return A;
}

// read the device scalars (synchronises the stream)
int pull_scalars(gpmood_t h) {
  CK(cudaMemcpyAsync(h->hsc, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

// the host's view after a step it waited for
void mark_synced(gpmood_t h) {
  h->sync_cur = h->cur;
  h->sync_nsteps = h->hsc->nsteps;
  h->pend = 0;
}

int step_error(gpmood_t h);
int step_launches(const gpmood_t h, int gated);

// wait for the queued asynchronous steps and settle the buffer rotation: the
// steps that ran are a prefix of those queued (the gate closes for good), and
// every successful one advanced the device's step count, so the rotation is
// the one at the last settle advanced by that count.  A failed step leaves
// the rotation, the time and the count where they were.  Returns a CUDA
// error only; a step error stays latched in the device scalars and in
// last_status.
int settle(gpmood_t h) {
  if (!h->pend) return 0;
  int rc = pull_scalars(h);
  if (rc) return rc;
  const long long m = h->hsc->nsteps - h->sync_nsteps;
  const int nb = h->sch.nbuf;
  h->cur = (int)((h->sync_cur + (m % nb) * h->sch.advance) % nb);
  h->launches = step_launches(h, 1);
  mark_synced(h);
  const int e = step_error(h);
  h->last_status = e;
  return 0;
}

void write_control(gpmood_t h, double cfl, double fixed_dt, int clip, double t_end,
                   double* tape = nullptr, uint8_t* otape = nullptr, void* stape = nullptr) {
  h->ctl.tape = tape;
  h->ctl.otape = otape;
  h->ctl.stape = stape;
  h->ctl.cfl = cfl;
  h->ctl.fixed_dt = fixed_dt;
  h->ctl.clip = clip;
  h->ctl.t_end = t_end;
  h->ctl.max_iters = h->max_iters;
}

int push_control(gpmood_t h) {
  // pageable source: staged by the CUDA driver at the call, so the host copy may
  // change right after
  CK(cudaMemcpyAsync(&h->sc->ctl, &h->ctl, sizeof(Control), cudaMemcpyHostToDevice, h->stream));
  h->ctl_dev = h->ctl;
  h->ctl_valid = 1;
  return 0;
}

// the same, skipped when the device already holds these controls
int push_control_if_changed(gpmood_t h) {
  if (h->ctl_valid && memcmp(&h->ctl_dev, &h->ctl, sizeof(Control)) == 0) return 0;
  return push_control(h);
}

// kernels launched by one step: the gate of a gated graph (1), dt (2), the
// ghost fill of the first stage's input (1), per stage the face kernels, the
// update and the MOOD loop (which fills the next stage's ghosts), finish (1)
int step_base_launches(int nstages, int face_kernels, int gated) {
  return (gated ? 1 : 0) + 2 + 1 + nstages * (2 + face_kernels) + 1;
}
// first-pass face kernels a stage: 1 (fused, or 1D), 2 (split 2D)
int face_kernels(const gpmood_t h) { return (h->g.dim == 2 && h->split_faces) ? 2 : 1; }
int step_launches(const gpmood_t h, int gated) {
  return step_base_launches(h->sch.nstages, face_kernels(h), gated);
}

int step_error(gpmood_t h) {
  if (h->hsc->err & kErrDt) return set_err(h, GPMOOD_E_DT);
  if (h->hsc->err & kErrCap) return set_err(h, GPMOOD_E_MOOD_CAP);
  if (h->hsc->err & kErrSync) return set_err(h, GPMOOD_E_SYNC);
  return GPMOOD_OK;
}

template <class Real>
MoodArgs mood_args(gpmood_t h) {
  MoodArgs M;
  M.queue[0] = h->queue[0];
  M.queue[1] = h->queue[1];
  M.stamp = h->stamp;
  M.stamp_stride = (long long)h->g.nx * h->g.ny;
  M.sc = h->sc;
  return M;
}

// the first-pass faces of both directions: one fused launch on 2D grids
// (split_faces = 0), else one launch per direction (x only in 1D)
template <class Real>
cudaError_t faces_both(gpmood_t h, const StageArgs<Real>& A, const ParityW<Real>& P,
                       cudaStream_t st) {
  if (h->g.dim == 2 && !h->split_faces) return Launch<Real>::faces_xy(h->cas.top, A, h->g, P, st);
  cudaError_t e = Launch<Real>::faces(h->cas.top, 0, A, h->g, P, st);
  if (e == cudaSuccess && h->g.dim == 2) e = Launch<Real>::faces(h->cas.top, 1, A, h->g, P, st);
  return e;
}

template <class Real>
int first_pass(gpmood_t h, const StageArgs<Real>& A, int ix, int s, const ParityW<Real>& P,
               const DirectW<Real>& D, cudaStream_t st) {
  // the later stages' inputs were filled by the previous stage's loop kernel
  if (s == 0) CK(launch_fill(h->U[ix], h->Uf[ix], h->g, h->sc, h->sch.st[s].tfrac, st));
  CK(faces_both<Real>(h, A, P, st));
  CK(Launch<Real>::update_first(A, h->g, h->det, D, st));
  return 0;
}

// the MOOD loop of stage s: one launch; a driver that refuses the
// cooperative launch gets a plain launch of the same co-resident grid from
// then on (the kernel's barrier waits are bounded either way)
template <class Real>
int mood_loop(gpmood_t h, const StageArgs<Real>& A, int s, const DirectW<Real>& D,
              cudaStream_t st) {
  const MoodArgs M = mood_args<Real>(h);
  // the loop kernel's tail: the ghost cells of the next stage's input (this
  // stage's output), or after the last stage the CFL rate of the new state
  LoopTail T;
  memset(&T, 0, sizeof(T));
  float* shadow = nullptr;  // the output's float shadow (FP32 path)
  if constexpr (sizeof(Real) == sizeof(float)) shadow = A.outr;
  if (s + 1 < h->sch.nstages) {
    T.X = A.out;
    T.Xf = shadow;
    T.tfrac = h->sch.st[s + 1].tfrac;
  } else {
    T.rate = 1;
    T.Xrate = A.out;
    T.Xfrate = shadow;
  }
  cudaError_t e = Launch<Real>::mood_loop(A, M, h->g, h->det, D, h->cas, s, T, h->mood_blocks,
                                          h->coop, st);
  if (e != cudaSuccess && h->coop) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      h->coop = 0;
      e = Launch<Real>::mood_loop(A, M, h->g, h->det, D, h->cas, s, T, h->mood_blocks, 0, st);
    }
  }
  CK(e);
  return 0;
}

// ---- eager step: stream launches, the host reads the scalars after every
// stage.  Used by gpmood_step_noalloc, which must not build graphs. ----
template <class Real>
int eager_stage(gpmood_t h, int s, int rot, const ParityW<Real>& P, const DirectW<Real>& D) {
  StageArgs<Real> A = stage_args<Real>(h, s, rot);
  const int ix = buf_of(h, rot, h->sch.st[s].in);
  int rc = first_pass<Real>(h, A, ix, s, P, D, h->stream);
  if (rc) return rc;
  rc = mood_loop<Real>(h, A, s, D, h->stream);
  if (rc) return rc;
  return pull_scalars(h);
}

// copy the interior of a ghosted state to an interior array (device)
int copy_interior(gpmood_t h, const double* Xg, double* out) {
  const Grid& g = h->g;
  for (int v = 0; v < 4; ++v)
    CK(cudaMemcpy2DAsync(out + (size_t)v * g.nx * g.ny, sizeof(double) * g.nx,
                         Xg + v * g.vstride + (size_t)g.H * g.pitch + g.H,
                         sizeof(double) * g.pitch, sizeof(double) * g.nx, g.ny,
                         cudaMemcpyDeviceToDevice, h->stream));
  return 0;
}

// the eager step; with a tape it also records the three stage inputs
// (interior, [3][4][ny][nx]) and the final radii of the three stages
int do_step(gpmood_t h, double cfl, double fixed_dt, int clip, double t_end,
            double* tape = nullptr, uint8_t* otape = nullptr, void* stape = nullptr) {
  if (!h->has_state) return set_err(h, GPMOOD_E_NOSTATE);
  g_pdl = h->pdl;
  const int a = h->cur;
  // the face kernels write the state tape (if any) themselves
  write_control(h, cfl, fixed_dt, clip, t_end, nullptr, nullptr, stape);
  int rc = push_control(h);
  if (rc) return rc;
  CK(launch_dt(h->U[a], h->Uf[a], h->g, h->sc, h->stream));
  const size_t nc = (size_t)h->g.nx * h->g.ny;
  for (int s = 0; s < h->sch.nstages; ++s) {
    if (tape) {
      rc = copy_interior(h, h->U[buf_of(h, a, h->sch.st[s].in)], tape + (size_t)s * 4 * nc);
      if (rc) return rc;
    }
    rc = h->precision == GPMOOD_FP32 ? eager_stage<float>(h, s, a, h->pw32, h->dw32)
                                     : eager_stage<double>(h, s, a, h->pw64, h->dw64);
    if (rc) return rc;
    rc = step_error(h);
    if (rc) return rc;
    if (otape) CK(cudaMemcpyAsync(otape + s * nc, h->ord + s * nc, nc, cudaMemcpyDeviceToDevice,
                                  h->stream));
  }
  CK(launch_finish(h->sc, step_base_launches(h->sch.nstages, face_kernels(h), 0), h->stream));
  rc = pull_scalars(h);
  if (rc) return rc;
  h->launches = step_launches(h, 0);
  h->cur = buf_of(h, a, h->sch.advance);
  mark_synced(h);
  h->last_status = GPMOOD_OK;
  return GPMOOD_OK;
}

// ---- graph step: one captured graph per buffer rotation; the MOOD loop of
// every stage iterates inside its kernel, so a step needs no host round trip ----
void rec_event(gpmood_t h, int prof, int cls, int open, cudaStream_t st) {
  if (!prof) return;
  int k = h->gev_n;
  cudaEventRecordWithFlags(h->gev[k], st, cudaEventRecordExternal);
  if (!open) h->gev_cls[(k - 1) / 2] = cls;
  h->gev_n = k + 1;
}

template <class Real>
int capture_stage(gpmood_t h, int s, int rot, const ParityW<Real>& P, const DirectW<Real>& D,
                  int prof, int record, cudaStream_t st) {
  StageArgs<Real> A = stage_args<Real>(h, s, rot);
  const int ix = buf_of(h, rot, h->sch.st[s].in);
  if (record) {
    k_tape_state<<<152 * 4, 256, 0, st>>>(h->U[ix], h->g, h->sc, s);
    CK(cudaGetLastError());
  }
  // the later stages' inputs were filled by the previous stage's loop kernel
  rec_event(h, prof, GPMOOD_K_GHOST, 1, st);
  if (s == 0) CK(launch_fill(h->U[ix], h->Uf[ix], h->g, h->sc, h->sch.st[s].tfrac, st));
  rec_event(h, prof, GPMOOD_K_GHOST, 0, st);
  if (h->g.dim == 2 && !h->split_faces) {
    // both directions in one kernel, timed as the x-face class
    rec_event(h, prof, GPMOOD_K_FACES_X, 1, st);
    CK(Launch<Real>::faces_xy(h->cas.top, A, h->g, P, st));
    rec_event(h, prof, GPMOOD_K_FACES_X, 0, st);
  } else {
    rec_event(h, prof, GPMOOD_K_FACES_X, 1, st);
    CK(Launch<Real>::faces(h->cas.top, 0, A, h->g, P, st));
    rec_event(h, prof, GPMOOD_K_FACES_X, 0, st);
    rec_event(h, prof, GPMOOD_K_FACES_Y, 1, st);
    if (h->g.dim == 2) CK(Launch<Real>::faces(h->cas.top, 1, A, h->g, P, st));
    rec_event(h, prof, GPMOOD_K_FACES_Y, 0, st);
  }
  rec_event(h, prof, GPMOOD_K_UPDATE, 1, st);
  CK(Launch<Real>::update_first(A, h->g, h->det, D, st));
  rec_event(h, prof, GPMOOD_K_UPDATE, 0, st);
  rec_event(h, prof, GPMOOD_K_MOOD, 1, st);
  int rc = mood_loop<Real>(h, A, s, D, st);
  if (rc) return rc;
  rec_event(h, prof, GPMOOD_K_MOOD, 0, st);
  if (record) {
    k_tape_ord<<<152, 256, 0, st>>>(A.ord, h->sc, s, (long long)h->g.nx * h->g.ny);
    CK(cudaGetLastError());
  }
  return 0;
}

// capture the step graph of rotation `cur`.  Plain graphs (gated = 1) put
// the whole step inside an IF node opened by k_step_gate, so that queued
// steps after an error or past t_end do nothing; profiled and recording
// graphs (read back after every step) have no gate.
int capture_step_impl(gpmood_t h, int cur, int prof, int record, int gated,
                      cudaGraphExec_t* out) {
  const int a = cur;
  cudaStream_t st = h->cs;
  h->gev_n = 0;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = 0;
  cudaStream_t bs = st;  // the stream the step body is captured on
  cudaGraphNode_t ifnode = nullptr;
  int body_open = 0;
  if (gated) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t graph;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle hif;
    cudaGraphNodeParams cp = {};
    if (cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, nullptr, nullptr, nullptr) !=
            cudaSuccess ||
        cudaGraphConditionalHandleCreate(&hif, graph, 0, cudaGraphCondAssignDefault) !=
            cudaSuccess ||
        launch_gate(h->sc, hif, st) != cudaSuccess ||
        cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, &deps, nullptr, &ndeps) !=
            cudaSuccess) {
      rc = GPMOOD_E_CUDA;
    } else {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = hif;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      if (cudaGraphAddNode(&ifnode, graph, deps, nullptr, ndeps, &cp) != cudaSuccess ||
          cudaStreamBeginCaptureToGraph(h->cs3, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                        0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        rc = GPMOOD_E_CUDA;
      else {
        bs = h->cs3;
        body_open = 1;
      }
    }
  }
  if (!rc) {
    rec_event(h, prof, GPMOOD_K_DT, 1, bs);
    if (launch_dt(h->U[a], h->Uf[a], h->g, h->sc, bs) != cudaSuccess) rc = GPMOOD_E_CUDA;
    rec_event(h, prof, GPMOOD_K_DT, 0, bs);
  }
  for (int s = 0; s < h->sch.nstages && !rc; ++s)
    rc = h->precision == GPMOOD_FP32
             ? capture_stage<float>(h, s, a, h->pw32, h->dw32, prof, record, bs)
             : capture_stage<double>(h, s, a, h->pw64, h->dw64, prof, record, bs);
  if (!rc &&
      launch_finish(h->sc, step_base_launches(h->sch.nstages, face_kernels(h), gated), bs) != cudaSuccess)
    rc = GPMOOD_E_CUDA;
  if (body_open) {
    cudaGraph_t tmp = nullptr;
    if (cudaStreamEndCapture(h->cs3, &tmp) != cudaSuccess) rc = rc ? rc : GPMOOD_E_CUDA;
    if (!rc && cudaStreamUpdateCaptureDependencies(st, &ifnode, nullptr, 1,
                                                   cudaStreamSetCaptureDependencies) !=
                   cudaSuccess)
      rc = GPMOOD_E_CUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (!rc && ee != cudaSuccess) rc = GPMOOD_E_CUDA;
  if (!rc && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) rc = GPMOOD_E_CUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  if (rc) return set_err(h, rc);
  if (prof) h->gev_pairs = h->gev_n / 2;
  return GPMOOD_OK;
}

int capture_step(gpmood_t h, int cur, int prof, int record, cudaGraphExec_t* out) {
  const int want_gate = !prof && !record && h->gated_ok >= 0;
  g_pdl = h->pdl;
  int rc = capture_step_impl(h, cur, prof, record, want_gate, out);
  if (rc && h->pdl) {
    // the CUDA driver refused programmatic edges in the step graph: plain
    // stream order from now on
    h->pdl = 0;
    g_pdl = 0;
    rc = capture_step_impl(h, cur, prof, record, want_gate, out);
  }
  if (rc && h->coop) {
    // the CUDA driver refused a cooperative kernel node: a plain launch of the
    // same co-resident grid
    h->coop = 0;
    rc = capture_step_impl(h, cur, prof, record, want_gate, out);
  }
  if (rc && want_gate && h->gated_ok == 0) {
    // the CUDA driver refused the gated graph: plain graphs without the gate, and
    // asynchronous steps run synchronously from now on
    h->gated_ok = -1;
    rc = capture_step_impl(h, cur, prof, record, 0, out);
  }
  if (!rc && want_gate) h->gated_ok = 1;
  if (!rc) h->last_status = GPMOOD_OK;
  return rc;
}

int graph_step(gpmood_t h, double cfl, double fixed_dt, int clip, double t_end,
               double* tape = nullptr, uint8_t* otape = nullptr, void* stape = nullptr) {
  if (!h->has_state) return set_err(h, GPMOOD_E_NOSTATE);
  int rc = settle(h);
  if (rc) return rc;
  if (h->eager) return do_step(h, cfl, fixed_dt, clip, t_end, tape, otape, stape);
  const int record = tape ? 1 : 0;
  const int prof = (h->prof_on && !record) ? 1 : 0;
  cudaGraphExec_t& ge = h->gexec[h->cur][record ? 2 : prof];
  if (!ge) {
    rc = capture_step(h, h->cur, prof, record, &ge);
    if (rc) return rc;
  }
  const int gated = !record && !prof && h->gated_ok == 1;
  write_control(h, cfl, fixed_dt, clip, t_end, tape, otape, stape);
  rc = push_control(h);
  if (rc) return rc;
  CK(cudaGraphLaunch(ge, h->stream));
  rc = pull_scalars(h);
  if (rc) return rc;
  if (prof) {
    for (int k = 0; k < h->gev_pairs; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->gev[2 * k], h->gev[2 * k + 1]) == cudaSuccess)
        h->prof_ms[h->gev_cls[k]] += ms;
    }
    const int S = h->sch.nstages;
    h->prof_n[GPMOOD_K_DT] += 2;
    h->prof_n[GPMOOD_K_GHOST] += 1;
    h->prof_n[GPMOOD_K_FACES_X] += S;
    h->prof_n[GPMOOD_K_FACES_Y] += (h->g.dim == 2 && h->split_faces) ? S : 0;
    h->prof_n[GPMOOD_K_UPDATE] += S;
    h->prof_n[GPMOOD_K_MOOD] += S;
  }
  mark_synced(h);
  rc = step_error(h);
  if (rc) return rc;
  h->launches = step_launches(h, gated);
  h->cur = buf_of(h, h->cur, h->sch.advance);
  mark_synced(h);
  h->last_status = GPMOOD_OK;
  return GPMOOD_OK;
}

// queue one step without waiting (plain gated graphs).  Eager handles,
// profiled steps and handles whose driver refused the gate step
// synchronously instead.
int graph_step_async(gpmood_t h, double cfl, double fixed_dt, int clip, double t_end) {
  if (!h->has_state) return set_err(h, GPMOOD_E_NOSTATE);
  if (h->eager || h->prof_on || h->gated_ok < 0) return graph_step(h, cfl, fixed_dt, clip, t_end);
  cudaGraphExec_t& ge = h->gexec[h->cur][0];
  if (!ge) {
    int rc = capture_step(h, h->cur, 0, 0, &ge);
    if (rc) return rc;
    if (h->gated_ok < 0) return graph_step(h, cfl, fixed_dt, clip, t_end);
  }
  write_control(h, cfl, fixed_dt, clip, t_end);
  int rc = push_control_if_changed(h);
  if (rc) return rc;
  CK(cudaGraphLaunch(ge, h->stream));
  // assume the step runs; settle() corrects the rotation if it did not
  h->cur = buf_of(h, h->cur, h->sch.advance);
  h->pend += 1;
  return GPMOOD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers of the precision-independent kernels
// ---------------------------------------------------------------------------
namespace gpm {

thread_local int g_pdl = 0;

cudaError_t launch_fill(double* X, float* Xf, const Grid& g, const Scalars* sc, double tfrac,
                        cudaStream_t st) {
  long long n = (long long)g.ny * 2 * g.H + (long long)2 * g.H * (g.nx + 2 * g.H);
  int blocks = (int)((n + 255) / 256);
  return launch_k(k_fill_ghosts, dim3(blocks), dim3(256), st, X, Xf, g, sc, tfrac);
}

cudaError_t launch_dt(const double* X, const float* Xf, const Grid& g, Scalars* sc,
                      cudaStream_t st) {
  long long n = (long long)g.nx * g.ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  cudaError_t e = launch_k(k_dt_reduce, dim3(blocks), dim3(256), st, X, Xf, g, sc);
  if (e != cudaSuccess) return e;
  return launch_k(k_dt_finalize, dim3(1), dim3(32), st, sc);
}

cudaError_t launch_finish(Scalars* sc, int base, cudaStream_t st) {
  return launch_k(k_finish_step, dim3(1), dim3(32), st, sc, base);
}

cudaError_t launch_gate(Scalars* sc, cudaGraphConditionalHandle hif, cudaStream_t st) {
  return launch_k(k_step_gate, dim3(1), dim3(32), st, sc, hif);
}

}  // namespace gpm

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* gpmood_strerror(int code) {
  switch (code) {
    case GPMOOD_OK: return "ok";
    case GPMOOD_E_INVAL: return "invalid argument";
    case GPMOOD_E_CUDA: return "CUDA error";
    case GPMOOD_E_OOM: return "device allocation failed";
    case GPMOOD_E_WEIGHTS: return "GP covariance matrix not positive definite";
    case GPMOOD_E_MOOD_CAP: return "MOOD iteration cap reached";
    case GPMOOD_E_DT: return "time step not positive or not finite";
    case GPMOOD_E_NOSTATE: return "no state set";
    case GPMOOD_E_TOO_BIG: return "grid too large for the static scratch";
    case GPMOOD_E_SYNC: return "a grid-wide barrier of the MOOD loop timed out";
    default: return "unknown error";
  }
}

int gpmood_create(const gpmood_grid* grid, double gamma, int R_max, double ell,
                  const gpmood_options* opts, gpmood_t* out) {
  if (!out) return GPMOOD_E_INVAL;
  *out = nullptr;
  if (!grid || R_max < 0 || R_max > 3 || !(gamma > 1.0) || !(ell > 0.0)) return GPMOOD_E_INVAL;
  gpmood_options o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  // cascade
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
  const int H = R_max + 1 > 2 ? R_max + 1 : 2;
  const int minn = H > 3 ? H : 3;
  if (grid->dim != 0 && grid->dim != 1 && grid->dim != 2) return GPMOOD_E_INVAL;
  const bool one_d = grid->dim == 1;
  if (grid->nx < minn || (one_d ? grid->ny != 1 : grid->ny < minn)) return GPMOOD_E_INVAL;
  if (!(grid->x1 > grid->x0) || (!one_d && !(grid->y1 > grid->y0))) return GPMOOD_E_INVAL;
  for (int s = 0; s < (one_d ? 2 : 4); ++s) {
    int k = grid->bc[s];
    if (k < 0 || k > 6) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_JET && s < 2) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_DMR_BOTTOM && s != 2) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_DMR_TOP && s != 3) return GPMOOD_E_INVAL;
  }
  if ((grid->bc[0] == 0) != (grid->bc[1] == 0)) return GPMOOD_E_INVAL;
  if (!one_d && (grid->bc[2] == 0) != (grid->bc[3] == 0)) return GPMOOD_E_INVAL;
  if (o.precision != GPMOOD_FP64 && o.precision != GPMOOD_FP32) return GPMOOD_E_INVAL;
  if (o.rk != 0 && o.rk != 3 && o.rk != 4) return GPMOOD_E_INVAL;
  if (o.riemann != 0 && o.riemann != 1) return GPMOOD_E_INVAL;
  if (o.recon != 0 && o.recon != 1) return GPMOOD_E_INVAL;
  if (o.recon == 1 && R_max != 1) return GPMOOD_E_INVAL;  // POL-MOOD3: Poly3 -> FOG

  gpmood_t h = new (std::nothrow) gpmood_s;
  if (!h) return GPMOOD_E_OOM;
  memset(h, 0, sizeof(*h));
  make_scheme(o.rk, &h->sch);
  const int S = h->sch.nstages;
  Grid& g = h->g;
  g.nx = grid->nx;
  g.ny = grid->ny;
  g.dim = one_d ? 1 : 2;
  g.H = H;
  g.pitch = round_up(g.nx + 2 * H, 32);
  g.gy = g.ny + 2 * H;
  g.vstride = (long long)g.pitch * g.gy;
  g.dx = (grid->x1 - grid->x0) / g.nx;
  g.dy = one_d ? g.dx : (grid->y1 - grid->y0) / g.ny;
  g.inv_dx = 1.0 / g.dx;
  g.inv_dy = 1.0 / g.dy;
  g.x0 = grid->x0;
  g.y0 = one_d ? 0.0 : grid->y0;
  g.gamma = gamma;
  for (int s = 0; s < 4; ++s) {
    // 1D: the ghost rows copy the single row (no y faces read them)
    g.bc[s] = (one_d && s >= 2) ? GPMOOD_BC_OUTFLOW : grid->bc[s];
    prim_to_cons(grid->bc_prim[s], gamma, g.bcU[s]);
  }
  g.periodic_x = grid->bc[0] == GPMOOD_BC_PERIODIC;
  g.periodic_y = g.bc[2] == GPMOOD_BC_PERIODIC;
  prim_to_cons(grid->dmr_post, gamma, g.dmr_post);
  prim_to_cons(grid->dmr_pre, gamma, g.dmr_pre);
  g.dmr_wall_x0 = grid->dmr_wall_x0;
  g.dmr_xs0 = grid->dmr_xs0;
  g.dmr_xs_speed = grid->dmr_xs_speed;
  g.jet_x0 = grid->jet_x0;
  g.jet_x1 = grid->jet_x1;
  prim_to_cons(grid->jet_prim[0], gamma, g.jetU[0]);
  prim_to_cons(grid->jet_prim[1], gamma, g.jetU[1]);
  g.riemann = o.riemann;
  g.rate_floor = jet_rate(g);

  for (int r = 0; r < 4; ++r) h->cas.next[r] = h->cas.prev[r] = r;
  for (int k = 0; k + 1 < nc; ++k) {
    h->cas.next[cascade[k]] = cascade[k + 1];
    h->cas.prev[cascade[k + 1]] = cascade[k];
  }
  h->cas.top = R_max;
  h->det.sigma_v = o.sigma_v > 0 ? o.sigma_v : 5.0;
  h->det.sigma_p = o.sigma_p > 0 ? o.sigma_p : 5.0;
  h->det.csd_on = o.csd_off ? 0 : 1;
  h->det.plateau_thr = fmin(g.dx * g.dx * g.dx, g.dy * g.dy * g.dy);
  h->det.delta = fmin(g.dx, g.dy);
  detect_derive(h->det, g);
  h->precision = o.precision;
  h->eager = o.eager ? 1 : 0;
  h->pdl = o.serial_launch ? 0 : 1;
  h->split_faces = o.split_faces ? 1 : 0;
  if ((h->precision == GPMOOD_FP32 ? Launch<float>::prepare() : Launch<double>::prepare()) !=
      cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GPMOOD_E_CUDA;
  }
  h->coop = 1;
  h->mood_blocks = h->precision == GPMOOD_FP32 ? Launch<float>::mood_loop_blocks()
                                               : Launch<double>::mood_loop_blocks();
  if (h->mood_blocks <= 0) {
    delete h;
    return GPMOOD_E_CUDA;
  }
  // a safety net only: radii never rise, so the loop ends; chains of
  // re-detected neighbours can take O(grid width) iterations
  h->max_iters = o.max_mood_iters > 0 ? o.max_mood_iters
                                      : 64 + 4 * (grid->nx > grid->ny ? grid->nx : grid->ny);

  // weights of every radius of the cascade, binary128 -> double / float:
  // GP, or Poly3 on the R = 1 rung of POL-MOOD3
  const bool poly3 = o.recon == 1;
  gpw_radius wr[4];
  memset(wr, 0, sizeof(wr));
  for (int k = 0; k < nc; ++k) {
    int R = cascade[k];
    if (R == 0) continue;
    int rc;
    if (poly3) rc = one_d ? gpw_poly3_1d(&wr[R]) : gpw_poly3(&wr[R]);
    else rc = one_d ? gpw_solve_1d(R, g.dx, ell, &wr[R]) : gpw_solve(R, g.dx, g.dy, ell, &wr[R]);
    if (rc != 0) {
      delete h;
      return GPMOOD_E_WEIGHTS;
    }
  }
  int da[25], db[25];
  double d2x[25], d2y[25];
  const int nd2 =
      poly3 ? gpw_second_derivative_poly3(one_d ? 1 : 0, g.dx, g.dy, da, db, d2x, d2y)
      : one_d ? gpw_second_derivative_1d(g.dx, ell, da, db, d2x, d2y)
              : gpw_second_derivative(g.dx, g.dy, ell, da, db, d2x, d2y);
  if (nd2 != 5) {
    delete h;
    return GPMOOD_E_WEIGHTS;
  }
  fill_weights<double>(wr, R_max, d2x, d2y, h->pw64, h->dw64);
  fill_weights<float>(wr, R_max, d2x, d2y, h->pw32, h->dw32);

  // device buffers
  const size_t ncell = (size_t)g.nx * g.ny;
  const size_t fsz = sizeof(double);  // face fluxes are FP64 on both paths
  bool ok = true;
  for (int k = 0; k < h->sch.nbuf; ++k)
    ok = ok && cudaMalloc(&h->U[k], sizeof(double) * 4 * (size_t)g.vstride) == cudaSuccess;
  if (h->precision == GPMOOD_FP32)
    for (int k = 0; k < h->sch.nbuf; ++k)
      ok = ok && cudaMalloc(&h->Uf[k], sizeof(float) * 4 * (size_t)g.vstride) == cudaSuccess;
  ok = ok && cudaMalloc(&h->Fx, fsz * 4 * (size_t)g.ny * (g.nx + 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->Fy, fsz * 4 * (size_t)(g.ny + 1) * g.nx) == cudaSuccess;
  const size_t nfb = (size_t)(g.nx + 1) * g.ny + (size_t)g.nx * (g.ny + 1);
  ok = ok && cudaMalloc(&h->fb, nfb) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ord, S * ncell) == cudaSuccess;
  ok = ok && cudaMalloc(&h->first, S * ncell) == cudaSuccess;
  ok = ok && cudaMalloc(&h->stamp, 2 * sizeof(uint32_t) * ncell) == cudaSuccess;
  ok = ok && cudaMalloc(&h->queue[0], sizeof(int) * ncell) == cudaSuccess;
  ok = ok && cudaMalloc(&h->queue[1], sizeof(int) * ncell) == cudaSuccess;
  ok = ok && cudaMalloc(&h->sc, sizeof(Scalars)) == cudaSuccess;
  ok = ok && cudaMallocHost(&h->hsc, sizeof(Scalars)) == cudaSuccess;
  if (!ok) {
    free_all(h);
    delete h;
    cudaGetLastError();
    return GPMOOD_E_OOM;
  }
  // the face fluxes start at zero: in 1D the y fluxes stay zero
  ok = cudaMemset(h->Fx, 0, fsz * 4 * (size_t)g.ny * (g.nx + 1)) == cudaSuccess &&
       cudaMemset(h->Fy, 0, fsz * 4 * (size_t)(g.ny + 1) * g.nx) == cudaSuccess &&
       cudaMemset(h->fb, 0, nfb) == cudaSuccess && cudaMemset(h->stamp, 0, 2 * sizeof(uint32_t) * ncell) == cudaSuccess &&
       cudaMemset(h->ord, 0, S * ncell) == cudaSuccess &&
       cudaMemset(h->first, 0, S * ncell) == cudaSuccess;
  for (int k = 0; k < h->sch.nbuf && ok; ++k)
    ok = cudaMemset(h->U[k], 0, sizeof(double) * 4 * (size_t)g.vstride) == cudaSuccess &&
         (!h->Uf[k] || cudaMemset(h->Uf[k], 0, sizeof(float) * 4 * (size_t)g.vstride) ==
                           cudaSuccess);
  if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
    free_all(h);
    delete h;
    return GPMOOD_E_CUDA;
  }
  bool evok = cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->cs2, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->cs3, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 64 && evok; ++k) evok = cudaEventCreate(&h->gev[k]) == cudaSuccess;
  if (!evok) {
    free_all(h);
    delete h;
    return GPMOOD_E_CUDA;
  }
  h->stream = nullptr;
  h->last_status = GPMOOD_OK;
  *out = h;
  return GPMOOD_OK;
}

int gpmood_set_stream(gpmood_t h, void* stream) {
  if (!h) return GPMOOD_E_INVAL;
  int rc = settle(h);  // queued steps finish on the old stream
  if (rc) return rc;
  h->stream = (cudaStream_t)stream;
  return GPMOOD_OK;
}

int gpmood_set_state(gpmood_t h, const double* U, int on_device) {
  if (!h || !U) return GPMOOD_E_INVAL;
  const Grid& g = h->g;
  h->cur = 0;
  const double* src = device_view(U, on_device);
  if (src) {
    // one kernel reads the cell averages (device memory, or pinned host
    // memory straight over the chip-to-chip link) into the ghosted layout
    // and the float shadow
    k_set_interior<<<152 * 8, 256, 0, h->stream>>>(src, h->U[0], h->Uf[0], g);
    CK(cudaGetLastError());
  } else {
    // pageable host memory: staged copies by the CUDA driver
    for (int v = 0; v < 4; ++v) {
      double* dst = h->U[0] + v * g.vstride + (size_t)g.H * g.pitch + g.H;
      const double* s = U + (size_t)v * g.nx * g.ny;
      CK(cudaMemcpy2DAsync(dst, sizeof(double) * g.pitch, s, sizeof(double) * g.nx,
                           sizeof(double) * g.nx, g.ny, cudaMemcpyHostToDevice, h->stream));
    }
    if (h->Uf[0]) {
      k_to_real<float><<<152 * 8, 256, 0, h->stream>>>(h->U[0], h->Uf[0], 4 * g.vstride);
      CK(cudaGetLastError());
    }
  }
  // MOOD stamps restart with the scalars
  CK(cudaMemsetAsync(h->stamp, 0, 2 * sizeof(uint32_t) * (size_t)g.nx * g.ny, h->stream));
  Scalars z;
  memset(&z, 0, sizeof(z));
  z.rate_bits = 0ull;
  *h->hsc = z;
  CK(cudaMemcpyAsync(h->sc, h->hsc, sizeof(Scalars), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->has_state = 1;
  h->pend = 0;  // queued steps (if any) ran before the copies above
  h->sync_cur = 0;
  h->sync_nsteps = 0;
  h->ctl_valid = 0;  // the device controls were zeroed with the scalars
  return GPMOOD_OK;
}

int gpmood_set_time(gpmood_t h, double t) {
  if (!h || !isfinite(t)) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&h->sc->t, &t, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GPMOOD_OK;
}

int gpmood_get_state(gpmood_t h, double* U, int on_device) {
  if (!h || !U) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  const Grid& g = h->g;
  double* dst = const_cast<double*>(device_view(U, on_device));
  if (dst) {
    k_get_interior<<<152 * 8, 256, 0, h->stream>>>(h->U[h->cur], dst, g);
    CK(cudaGetLastError());
  } else {
    for (int v = 0; v < 4; ++v) {
      const double* s = h->U[h->cur] + v * g.vstride + (size_t)g.H * g.pitch + g.H;
      CK(cudaMemcpy2DAsync(U + (size_t)v * g.nx * g.ny, sizeof(double) * g.nx, s,
                           sizeof(double) * g.pitch, sizeof(double) * g.nx, g.ny,
                           cudaMemcpyDeviceToHost, h->stream));
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return GPMOOD_OK;
}

int gpmood_step(gpmood_t h, double cfl, double* dt_out) {
  if (!h || !(cfl > 0.0)) return GPMOOD_E_INVAL;
  int rc = graph_step(h, cfl, 0.0, 0, 0.0);
  if (rc) return rc;
  if (dt_out) *dt_out = h->hsc->dt;
  return GPMOOD_OK;
}

int gpmood_step_dt(gpmood_t h, double dt) {
  if (!h || !(dt > 0.0)) return GPMOOD_E_INVAL;
  return graph_step(h, 1.0, dt, 0, 0.0);
}

int gpmood_step_async(gpmood_t h, double cfl) {
  if (!h || !(cfl > 0.0)) return GPMOOD_E_INVAL;
  return graph_step_async(h, cfl, 0.0, 0, 0.0);
}

int gpmood_sync(gpmood_t h) {
  if (!h) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  rc = pull_scalars(h);
  if (rc) return rc;
  return step_error(h);
}

int gpmood_launch_count(gpmood_t h, long long* count) {
  if (!h || !count) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  rc = pull_scalars(h);
  if (rc) return rc;
  *count = h->hsc->launches;
  return GPMOOD_OK;
}

// steps clipped to t_end.  Graph handles queue them in chunks sized from the
// last time step and wait once per chunk; the gate turns the steps queued
// past t_end into no-ops.
int gpmood_run(gpmood_t h, double t_end, double cfl, long long* nsteps_out) {
  if (!h || !(cfl > 0.0)) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  rc = pull_scalars(h);
  if (rc) return rc;
  const long long n0 = h->hsc->nsteps;
  const double stop = t_end * (1.0 - 1e-14);
  while (h->hsc->t < stop) {
    const double t = h->hsc->t, dt = h->hsc->dt;
    long long est = 1;
    if (dt > 0.0 && isfinite(dt)) est = (long long)ceil((t_end - t) / dt) + 1;
    const int chunk = (int)(est < 1 ? 1 : (est > 64 ? 64 : est));
    for (int k = 0; k < chunk; ++k) {
      rc = graph_step_async(h, cfl, 0.0, 1, t_end);
      if (rc) return rc;
      // a step taken synchronously (eager or profiled handles) has updated
      // the host scalars: stop at t_end as the device gate would
      if (!h->pend && !(h->hsc->t < stop)) break;
    }
    rc = settle(h);
    if (rc) return rc;
    rc = pull_scalars(h);
    if (rc) return rc;
    rc = step_error(h);
    if (rc) return rc;
  }
  if (nsteps_out) *nsteps_out = h->hsc->nsteps - n0;
  return GPMOOD_OK;
}

int gpmood_flags(gpmood_t h, uint8_t* order_out, uint8_t* first_out, gpmood_stats* stats_out) {
  if (!h) return GPMOOD_E_INVAL;
  int rc0 = settle(h);
  if (rc0) return rc0;
  const size_t nc = (size_t)h->g.nx * h->g.ny;
  const size_t S = (size_t)h->sch.nstages;
  if (order_out) CK(cudaMemcpyAsync(order_out, h->ord, S * nc, cudaMemcpyDeviceToHost, h->stream));
  if (first_out) CK(cudaMemcpyAsync(first_out, h->first, S * nc, cudaMemcpyDeviceToHost, h->stream));
  int rc = pull_scalars(h);
  if (rc) return rc;
  if (stats_out) {
    const Scalars& s = *h->hsc;
    stats_out->t = s.t;
    stats_out->dt = s.dt;
    stats_out->nsteps = s.nsteps;
    for (int k = 0; k < 5; ++k) {
      stats_out->iters[k] = s.iters[k];
      stats_out->nbad_first[k] = s.nbad_first[k];
      stats_out->nbad_total[k] = s.nbad_total[k];
      stats_out->nfog_pad[k] = s.nfog_pad[k];
    }
    stats_out->status = h->last_status;
  }
  return GPMOOD_OK;
}

int gpmood_destroy(gpmood_t h) {
  if (!h) return GPMOOD_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return GPMOOD_OK;
}

int gpmood_last_launches(gpmood_t h) { return h ? h->launches : 0; }

int gpmood_profile(gpmood_t h, int enable) {
  if (!h) return GPMOOD_E_INVAL;
  int rc = settle(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  h->prof_on = enable ? 1 : 0;
  if (enable)
    for (int k = 0; k < GPMOOD_NKCLASS; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  return GPMOOD_OK;
}

int gpmood_kernel_times(gpmood_t h, double* ms, long long* launches) {
  if (!h) return GPMOOD_E_INVAL;
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < GPMOOD_NKCLASS; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_n[k];
  }
  return GPMOOD_OK;
}

// ---------------------------------------------------------------------------
// recorded steps, replay with given radii, and the adjoint
// ---------------------------------------------------------------------------
int gpmood_step_record(gpmood_t h, double cfl, double dt_fixed, double* tape, uint8_t* otape,
                       double* dt_out) {
  return gpmood_step_record_states(h, cfl, dt_fixed, tape, otape, nullptr, dt_out);
}

int gpmood_step_record_states(gpmood_t h, double cfl, double dt_fixed, double* tape,
                              uint8_t* otape, void* stape, double* dt_out) {
  if (!h || !tape || !otape || (!(cfl > 0.0) && !(dt_fixed > 0.0))) return GPMOOD_E_INVAL;
  if (h->sch.nstages != 3) return GPMOOD_E_INVAL;  // the adjoint follows SSP-RK3
  if (stape && h->g.dim != 2) return GPMOOD_E_INVAL;
  int rc = graph_step(h, cfl > 0.0 ? cfl : 1.0, dt_fixed > 0.0 ? dt_fixed : 0.0, 0, 0.0, tape,
                      otape, stape);
  if (rc) return rc;
  if (dt_out) *dt_out = h->hsc->dt;
  return GPMOOD_OK;
}

int gpmood_state_tape_bytes(gpmood_t h, size_t* bytes) {
  if (!h || !bytes) return GPMOOD_E_INVAL;
  const Grid& g = h->g;
  const size_t nf = (size_t)(g.nx + 1) * g.ny + (size_t)g.nx * (g.ny + 1);
  const size_t qt = (size_t)rule_q(h->cas.top);
  const size_t real = h->precision == GPMOOD_FP32 ? sizeof(float) : sizeof(double);
  *bytes = (size_t)h->sch.nstages * 8 * qt * nf * real;
  return GPMOOD_OK;
}

}  // extern "C"

namespace {

template <class Real>
int frozen_step(gpmood_t h, const uint8_t* otape, double dt, const DirectW<Real>& D) {
  const int a = h->cur;
  g_pdl = h->pdl;
  write_control(h, 1.0, dt, 0, 0.0);
  int rc = push_control(h);
  if (rc) return rc;
  CK(launch_dt(h->U[a], h->Uf[a], h->g, h->sc, h->stream));
  const size_t nc = (size_t)h->g.nx * h->g.ny;
  for (int s = 0; s < h->sch.nstages; ++s) {
    const int ix = buf_of(h, a, h->sch.st[s].in);
    CK(launch_fill(h->U[ix], h->Uf[ix], h->g, h->sc, h->sch.st[s].tfrac, h->stream));
    StageArgs<Real> A = stage_args<Real>(h, s, a);
    CK(cudaMemcpyAsync(A.ord, otape + s * nc, nc, cudaMemcpyDeviceToDevice, h->stream));
    CK(LaunchA<Real>::frozen_stage(A, h->g, D, h->stream));
  }
  CK(launch_finish(h->sc, 0, h->stream));  // replay steps are not in the launch count
  rc = pull_scalars(h);
  if (rc) return rc;
  mark_synced(h);
  if (h->hsc->err & kErrDt) return set_err(h, GPMOOD_E_DT);
  h->cur = buf_of(h, a, h->sch.advance);
  mark_synced(h);
  return GPMOOD_OK;
}

int adj_buffers(gpmood_t h) {
  if (h->aX) return 0;
  const Grid& g = h->g;
  const size_t nc = (size_t)g.nx * g.ny;
  const size_t rs = h->precision == GPMOOD_FP32 ? sizeof(float) : sizeof(double);
  h->ax.nf = (long long)(g.nx + 1) * g.ny;
  h->ay.nf = (long long)g.nx * (g.ny + 1);
  bool ok = cudaMalloc(&h->aX, sizeof(double) * 4 * (size_t)g.vstride) == cudaSuccess &&
            cudaMalloc(&h->aXr, rs * 4 * (size_t)g.vstride) == cudaSuccess &&
            cudaMalloc(&h->aG, sizeof(double) * 4 * (size_t)g.vstride) == cudaSuccess &&
            cudaMalloc(&h->av, sizeof(double) * 4 * nc) == cudaSuccess &&
            cudaMalloc(&h->aw, sizeof(double) * 4 * nc) == cudaSuccess &&
            cudaMalloc(&h->amu, sizeof(double) * 4 * nc) == cudaSuccess &&
            cudaMalloc(&h->ax.L, rs * 4 * kMaxQ * (size_t)h->ax.nf) == cudaSuccess &&
            cudaMalloc(&h->ax.R, rs * 4 * kMaxQ * (size_t)h->ax.nf) == cudaSuccess &&
            cudaMalloc(&h->ax.K, (size_t)h->ax.nf) == cudaSuccess &&
            cudaMalloc(&h->ay.L, rs * 4 * kMaxQ * (size_t)h->ay.nf) == cudaSuccess &&
            cudaMalloc(&h->ay.R, rs * 4 * kMaxQ * (size_t)h->ay.nf) == cudaSuccess &&
            cudaMalloc(&h->ay.K, (size_t)h->ay.nf) == cudaSuccess &&
            cudaMalloc(&h->aord, 3 * nc) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return set_err(h, GPMOOD_E_OOM);
  }
  CK(cudaMemset(h->aX, 0, sizeof(double) * 4 * (size_t)g.vstride));
  return 0;
}

// w = v - dt (dF/dX)^T v at the stage input X (interior) with radii ords
template <class Real>
int adj_stage(gpmood_t h, const double* X, const uint8_t* ords, double ts, double dt,
              const double* v, double* w, const ParityW<Real>& P, const DirectW<Real>& D,
              const void* st) {
  const Grid& g = h->g;
  if (st) {
    // the recorded face states: no reconstruction, no ghosted copy of X
    CK(LaunchA<Real>::adj_faces_stored(st, v, ords, g, P, D, h->ax, h->ay, h->stream));
    CK(LaunchA<Real>::adj_gather(g, D, h->ax, h->ay, h->aG, h->stream));
    k_adj_fold_y<<<(g.nx + 2 * g.H + 127) / 128, 128, 0, h->stream>>>(h->aG, g);
    k_adj_fold_x<<<(g.ny + 127) / 128, 128, 0, h->stream>>>(h->aG, g);
    k_adj_stage_out<<<152 * 8, 256, 0, h->stream>>>(w, v, h->aG, g, dt);
    CK(cudaGetLastError());
    return 0;
  }
  for (int c = 0; c < 4; ++c)
    CK(cudaMemcpy2DAsync(h->aX + c * g.vstride + (size_t)g.H * g.pitch + g.H,
                         sizeof(double) * g.pitch, X + (size_t)c * g.nx * g.ny,
                         sizeof(double) * g.nx, sizeof(double) * g.nx, g.ny,
                         cudaMemcpyDeviceToDevice, h->stream));
  const long long ngh = (long long)g.ny * 2 * g.H + 2LL * g.H * (g.nx + 2 * g.H);
  const int gb = (int)((ngh + 255) / 256);
  k_fill_ghosts_at<<<gb, 256, 0, h->stream>>>(h->aX, g, ts);
  CK(cudaGetLastError());
  CK(LaunchA<Real>::adj_faces(h->aX, h->aXr, v, ords, g, P, D, h->ax, h->ay, h->stream));
  CK(LaunchA<Real>::adj_gather(g, D, h->ax, h->ay, h->aG, h->stream));
  k_adj_fold_y<<<(g.nx + 2 * g.H + 127) / 128, 128, 0, h->stream>>>(h->aG, g);
  k_adj_fold_x<<<(g.ny + 127) / 128, 128, 0, h->stream>>>(h->aG, g);
  k_adj_stage_out<<<152 * 8, 256, 0, h->stream>>>(w, v, h->aG, g, dt);
  CK(cudaGetLastError());
  return 0;
}

template <class Real>
int step_adjoint(gpmood_t h, const double* tape, const uint8_t* otape, const void* stape,
                 double dt, double t, const double* lam, double* out, const ParityW<Real>& P,
                 const DirectW<Real>& D) {
  const size_t nc = (size_t)h->g.nx * h->g.ny, n4 = 4 * nc;
  // the state tape of stage s
  size_t sbytes = 0;
  gpmood_state_tape_bytes(h, &sbytes);
  auto st = [&](int s) -> const void* {
    return stape ? (const void*)((const char*)stape + s * (sbytes / 3)) : nullptr;
  };
  const int nb = 152 * 8;
  double *mu = h->amu, *v = h->av, *w = h->aw;
  // U^{n+1} = (U^n + 2 Y3)/3
  k_lincomb<<<nb, 256, 0, h->stream>>>(mu, 1.0 / 3.0, lam, 0.0, nullptr, (long long)n4);
  k_lincomb<<<nb, 256, 0, h->stream>>>(v, 2.0 / 3.0, lam, 0.0, nullptr, (long long)n4);
  // Y3 = X3 - dt F(X3), X3 = (3 U^n + Y2)/4
  int rc = adj_stage<Real>(h, tape + 2 * n4, otape + 2 * nc, t + 0.5 * dt, dt, v, w, P, D, st(2));
  if (rc) return rc;
  k_lincomb<<<nb, 256, 0, h->stream>>>(mu, 1.0, mu, 0.75, w, (long long)n4);
  k_lincomb<<<nb, 256, 0, h->stream>>>(v, 0.25, w, 0.0, nullptr, (long long)n4);
  // Y2 = X2 - dt F(X2), X2 = Y1
  rc = adj_stage<Real>(h, tape + n4, otape + nc, t + dt, dt, v, w, P, D, st(1));
  if (rc) return rc;
  // Y1 = X1 - dt F(X1), X1 = U^n
  rc = adj_stage<Real>(h, tape, otape, t, dt, w, v, P, D, st(0));
  if (rc) return rc;
  k_lincomb<<<nb, 256, 0, h->stream>>>(out, 1.0, mu, 1.0, v, (long long)n4);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return GPMOOD_OK;
}

}  // namespace

extern "C" {

int gpmood_step_frozen(gpmood_t h, const uint8_t* otape, double dt) {
  if (!h || !otape || !(dt > 0.0) || h->g.dim != 2 || h->sch.nstages != 3) return GPMOOD_E_INVAL;
  if (!h->has_state) return GPMOOD_E_NOSTATE;
  int rc = settle(h);
  if (rc) return rc;
  return h->precision == GPMOOD_FP32 ? frozen_step<float>(h, otape, dt, h->dw32)
                                     : frozen_step<double>(h, otape, dt, h->dw64);
}

int gpmood_step_adjoint(gpmood_t h, const double* tape, const uint8_t* otape, double dt, double t,
                        const double* lam_in, double* lam_out) {
  return gpmood_step_adjoint_states(h, tape, otape, nullptr, dt, t, lam_in, lam_out);
}

int gpmood_step_adjoint_states(gpmood_t h, const double* tape, const uint8_t* otape,
                               const void* stape, double dt, double t, const double* lam_in,
                               double* lam_out) {
  if (!h || !tape || !otape || !lam_in || !lam_out || !(dt > 0.0) || h->g.dim != 2 ||
      h->sch.nstages != 3 || h->g.riemann != 0)  // the reverse Riemann solver is HLLC's
    return GPMOOD_E_INVAL;
  int rc = settle(h);
  if (rc) return rc;
  rc = adj_buffers(h);
  if (rc) return rc;
  return h->precision == GPMOOD_FP32
             ? step_adjoint<float>(h, tape, otape, stape, dt, t, lam_in, lam_out, h->pw32,
                                   h->dw32)
             : step_adjoint<double>(h, tape, otape, stape, dt, t, lam_in, lam_out, h->pw64,
                                    h->dw64);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// gpmood_step_noalloc: the step on a temporary handle whose device buffers
// live in one file-scope device array.  In host code the array's name only
// stands for the symbol; the device address comes from
// cudaGetSymbolAddress, once per device, with that device current.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GPMOOD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices];

// device address of the scratch array on the current device
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GPMOOD_E_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GPMOOD_E_CUDA;
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return GPMOOD_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int gpmood_step_noalloc(const gpmood_grid* grid, double gamma, int R_max, double ell,
                                   const gpmood_options* opts, const double* U_in, double* U_out,
                                   double t, double cfl, double* dt_out, void* stream) {
  if (!grid || !U_in || !U_out || !(cfl > 0.0) || !isfinite(t)) return GPMOOD_E_INVAL;
  // two-dimensional grids only (0 is the default 2); other values are
  // refused as gpmood_create refuses them
  if (grid->dim != 0 && grid->dim != 2) return GPMOOD_E_INVAL;
  if (R_max < 0 || R_max > 3 || !(gamma > 1.0) || !(ell > 0.0)) return GPMOOD_E_INVAL;
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
  const int H = R_max + 1 > 2 ? R_max + 1 : 2;
  const int minn = H > 3 ? H : 3;
  if (grid->nx < minn || grid->ny < minn) return GPMOOD_E_INVAL;
  if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0)) return GPMOOD_E_INVAL;
  for (int s = 0; s < 4; ++s) {
    int k = grid->bc[s];
    if (k < 0 || k > 6) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_JET && s < 2) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_DMR_BOTTOM && s != 2) return GPMOOD_E_INVAL;
    if (k == GPMOOD_BC_DMR_TOP && s != 3) return GPMOOD_E_INVAL;
  }
  if ((grid->bc[0] == 0) != (grid->bc[1] == 0)) return GPMOOD_E_INVAL;
  if ((grid->bc[2] == 0) != (grid->bc[3] == 0)) return GPMOOD_E_INVAL;
  if (o.precision != GPMOOD_FP64 && o.precision != GPMOOD_FP32) return GPMOOD_E_INVAL;
  // SSP-RK3 only (0 is the default 3): the scratch holds three states
  if (o.rk != 0 && o.rk != 3) return GPMOOD_E_INVAL;
  if (o.riemann != 0 && o.riemann != 1) return GPMOOD_E_INVAL;
  if (o.recon != 0 && o.recon != 1) return GPMOOD_E_INVAL;
  if (o.recon == 1 && R_max != 1) return GPMOOD_E_INVAL;

  // the temporary handle lives on the host stack
  gpmood_s hs;
  gpmood_s* h = &hs;
  memset(h, 0, sizeof(*h));
  make_scheme(3, &h->sch);
  Grid& g = h->g;
  g.nx = grid->nx;
  g.dim = 2;
  g.ny = grid->ny;
  g.H = H;
  g.pitch = round_up(g.nx + 2 * H, 32);
  g.gy = g.ny + 2 * H;
  g.vstride = (long long)g.pitch * g.gy;

  // carve the buffers out of the scratch, 256-byte aligned each
  const size_t ncell = (size_t)g.nx * g.ny;
  const size_t fsz = sizeof(double);  // face fluxes are FP64 on both paths
  const size_t sz_state = align256(sizeof(double) * 4 * (size_t)g.vstride);
  const size_t sz_fx = align256(fsz * 4 * (size_t)g.ny * (g.nx + 1));
  const size_t sz_fy = align256(fsz * 4 * (size_t)(g.ny + 1) * g.nx);
  const size_t nfb = (size_t)(g.nx + 1) * g.ny + (size_t)g.nx * (g.ny + 1);
  const size_t sz_fb = align256(nfb), sz_c3 = align256(3 * ncell);
  const size_t sz_stamp = align256(2 * sizeof(uint32_t) * ncell);
  const size_t sz_q = align256(sizeof(int) * ncell);
  const size_t sz_sc = align256(sizeof(Scalars));
  const size_t sz_shadow =
      o.precision == GPMOOD_FP32 ? align256(sizeof(float) * 4 * (size_t)g.vstride) : 0;
  const size_t need = 3 * sz_state + 3 * sz_shadow + sz_fx + sz_fy + sz_fb + 2 * sz_c3 +
                      sz_stamp + 2 * sz_q + sz_sc;
  if (need > (size_t)GPMOOD_NOALLOC_SCRATCH_BYTES) return GPMOOD_E_TOO_BIG;

  g.dx = (grid->x1 - grid->x0) / g.nx;
  g.dy = (grid->y1 - grid->y0) / g.ny;
  g.inv_dx = 1.0 / g.dx;
  g.inv_dy = 1.0 / g.dy;
  g.x0 = grid->x0;
  g.y0 = grid->y0;
  g.gamma = gamma;
  for (int s = 0; s < 4; ++s) {
    g.bc[s] = grid->bc[s];
    prim_to_cons(grid->bc_prim[s], gamma, g.bcU[s]);
  }
  g.periodic_x = grid->bc[0] == GPMOOD_BC_PERIODIC;
  g.periodic_y = grid->bc[2] == GPMOOD_BC_PERIODIC;
  prim_to_cons(grid->dmr_post, gamma, g.dmr_post);
  prim_to_cons(grid->dmr_pre, gamma, g.dmr_pre);
  g.dmr_wall_x0 = grid->dmr_wall_x0;
  g.dmr_xs0 = grid->dmr_xs0;
  g.dmr_xs_speed = grid->dmr_xs_speed;
  g.jet_x0 = grid->jet_x0;
  g.jet_x1 = grid->jet_x1;
  prim_to_cons(grid->jet_prim[0], gamma, g.jetU[0]);
  prim_to_cons(grid->jet_prim[1], gamma, g.jetU[1]);
  g.riemann = o.riemann;
  g.rate_floor = jet_rate(g);
  for (int r = 0; r < 4; ++r) h->cas.next[r] = h->cas.prev[r] = r;
  for (int k = 0; k + 1 < nc; ++k) {
    h->cas.next[cascade[k]] = cascade[k + 1];
    h->cas.prev[cascade[k + 1]] = cascade[k];
  }
  h->cas.top = R_max;
  h->det.sigma_v = o.sigma_v > 0 ? o.sigma_v : 5.0;
  h->det.sigma_p = o.sigma_p > 0 ? o.sigma_p : 5.0;
  h->det.csd_on = o.csd_off ? 0 : 1;
  h->det.plateau_thr = fmin(g.dx * g.dx * g.dx, g.dy * g.dy * g.dy);
  h->det.delta = fmin(g.dx, g.dy);
  detect_derive(h->det, g);
  h->precision = o.precision;
  // a safety net only: radii never rise, so the loop ends; chains of
  // re-detected neighbours can take O(grid width) iterations
  h->max_iters = o.max_mood_iters > 0 ? o.max_mood_iters
                                      : 64 + 4 * (grid->nx > grid->ny ? grid->nx : grid->ny);
  h->split_faces = o.split_faces ? 1 : 0;
  if ((h->precision == GPMOOD_FP32 ? Launch<float>::prepare() : Launch<double>::prepare()) !=
      cudaSuccess)
    return GPMOOD_E_CUDA;
  h->coop = 1;
  h->mood_blocks = h->precision == GPMOOD_FP32 ? Launch<float>::mood_loop_blocks()
                                               : Launch<double>::mood_loop_blocks();
  if (h->mood_blocks <= 0) return GPMOOD_E_CUDA;

  // GP weights: binary128 solve on the host stack
  gpw_radius wr[4];
  memset(wr, 0, sizeof(wr));
  for (int k = 0; k < nc; ++k) {
    int R = cascade[k];
    if (R == 0) continue;
    const int rc = o.recon == 1 ? gpw_poly3(&wr[R]) : gpw_solve(R, g.dx, g.dy, ell, &wr[R]);
    if (rc != 0) return GPMOOD_E_WEIGHTS;
  }
  int da[25], db[25];
  double d2x[25], d2y[25];
  const int nd2 = o.recon == 1 ? gpw_second_derivative_poly3(0, g.dx, g.dy, da, db, d2x, d2y)
                               : gpw_second_derivative(g.dx, g.dy, ell, da, db, d2x, d2y);
  if (nd2 != 5) return GPMOOD_E_WEIGHTS;
  fill_weights<double>(wr, R_max, d2x, d2y, h->pw64, h->dw64);
  fill_weights<float>(wr, R_max, d2x, d2y, h->pw32, h->dw32);

  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  unsigned char* p = base;
  for (int k = 0; k < 3; ++k) {
    h->U[k] = (double*)p;
    p += sz_state;
  }
  for (int k = 0; k < 3 && sz_shadow; ++k) {
    h->Uf[k] = (float*)p;
    p += sz_shadow;
  }
  h->Fx = p; p += sz_fx;
  h->Fy = p; p += sz_fy;
  h->fb = p; p += sz_fb;
  h->ord = p; p += sz_c3;
  h->first = p; p += sz_c3;
  h->stamp = (uint32_t*)p; p += sz_stamp;
  h->queue[0] = (int*)p; p += sz_q;
  h->queue[1] = (int*)p; p += sz_q;
  h->sc = (Scalars*)p;
  // the host mirror of the scalars lives on this call's stack (pageable
  // memory, no allocation): calls on different devices or threads share no
  // host state
  Scalars host_sc;
  memset(&host_sc, 0, sizeof(host_sc));
  h->hsc = &host_sc;
  h->stream = (cudaStream_t)stream;

  // what the kernels expect to start at zero: face-CAD flags and MOOD stamps
  CK(cudaMemsetAsync(h->fb, 0, nfb, h->stream));
  CK(cudaMemsetAsync(h->stamp, 0, 2 * sizeof(uint32_t) * ncell, h->stream));
  rc = gpmood_set_state(h, U_in, 1);
  if (rc) return rc;
  if (t != 0.0) {
    rc = gpmood_set_time(h, t);
    if (rc) return rc;
  }
  // the eager driver: a captured graph would need driver allocations
  rc = do_step(h, cfl, 0.0, 0, 0.0);
  if (rc) return rc;
  if (dt_out) *dt_out = h->hsc->dt;
  return gpmood_get_state(h, U_out, 1);
}
