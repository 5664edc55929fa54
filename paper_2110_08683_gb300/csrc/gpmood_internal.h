// gpmood_internal.h -- types shared by the host driver and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpm {

constexpr int kNV = 4;        // conservative variables (rho, rho u, rho v, rho E)
constexpr int kMaxN = 25;     // stencil size of the largest radius (R = 3)
constexpr int kMaxQ = 4;      // Gauss points of the largest radius
constexpr int kSegCells = 32; // cells per warp segment in the face kernels
constexpr int kSegFaces = kSegCells - 1;
constexpr int kFaceWarps = 8; // warps per face-kernel block

// programmatic dependent launch: a step kernel launched while its
// predecessor drains waits here, before touching memory, until the
// predecessor has completed and its writes are visible (a no-op without the
// launch attribute); pdl_trigger lets the successor be scheduled early
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// geometry and boundary data, passed by value to every kernel
struct Grid {
  int nx, ny, H;          // interior cells and ghost layers
  int dim;                // 2, or 1 (ny = 1, x faces only)
  int pitch, gy;          // ghosted row length (elements) and ghosted rows
  long long vstride;      // elements per variable plane of a ghosted state
  double dx, dy, inv_dx, inv_dy;
  double x0, y0;
  double gamma;
  int bc[4];              // W, E, S, N
  int periodic_x, periodic_y;
  double bcU[4][4];       // conservative Dirichlet state per side
  double dmr_post[4], dmr_pre[4];  // conservative states
  double dmr_wall_x0, dmr_xs0, dmr_xs_speed;
  double jet_x0, jet_x1;  // inflow slit of the JET kind
  double jetU[2][4];      // conservative jet states, S and N sides
  int riemann;            // 0 HLLC, 1 HLL
  double rate_floor;      // CFL rate of the jet inflow states (0: no jet side)
};

// step controls written by the host before every step
struct Control {
  double cfl;        // CFL number of the step
  double fixed_dt;   // > 0: take this step instead of the CFL one
  double t_end;      // clip target when clip != 0
  int clip;
  int max_iters;     // MOOD iteration cap per stage
  double* tape;      // recorded steps: stage inputs [3][4][ny][nx] (or null)
  uint8_t* otape;    // and the final radii [3][ny][nx]
  void* stape;       // and the reconstructed face states (Real, or null): per stage
                     // x faces left, x right, y lower, y upper, each [4][q_top][faces]
};

// scalars living on the device (one per handle)
struct Scalars {
  Control ctl;
  double t;                     // time at the start of the current step
  double dt;                    // current step
  unsigned long long rate_bits;  // running max of the CFL rate (|u|+c)/dx as ordered bits
  int err;                      // error bits (kErr*)
  int count[2];                 // queue lengths (double buffered)
  int slot;                     // queue holding the cells to work on
  int go;                       // MOOD loop continues (mirrors the graph condition)
  unsigned int stamp_cur;       // stamp of the cells in the current queue
  int iters[5], nbad_first[5], nbad_total[5], nfog_pad[5];  // per RK stage
  long long nsteps;
  long long launches;           // kernels launched by graph steps since the state was set
  int nactive;                  // batches: problems still advancing in this step
  unsigned int bar_count;       // grid barrier of the MOOD loop kernel: arrivals
  unsigned int bar_gen;         // and generation (count returns to 0 after each use)
  int rate_ready;               // rate_bits holds the CFL rate of the current state
  int rate_bad;                 // and that state had a cell with no admissible rate
};

// work the MOOD loop kernel of a stage does once its loop has ended, while its
// grid is resident: fill the ghost cells of the stage's output, which the
// next stage reads (X, and its float shadow Xf on the FP32 path, at time
// t + tfrac dt), and, after the last stage, reduce the CFL rate of the new
// state for the next step's time step
struct LoopTail {
  double* X;     // null: no ghost fill
  float* Xf;
  double tfrac;
  int rate;      // 1: the rate of X_rate (and its shadow) into Scalars::rate_bits
  const double* Xrate;
  const float* Xfrate;
};

constexpr int kErrDt = 1;       // non-finite or non-positive time step
constexpr int kErrCap = 2;      // MOOD iteration cap reached
constexpr int kErrSync = 4;     // a grid barrier of the MOOD loop kernel gave up waiting

// parity-decomposed prediction weights of one radius for the first pass
// (see the stencil-symmetry note in the face kernels)
template <class Real>
struct ParityW {
  Real cx[2][kMaxN];  // x faces (east-face weights), per g slot, per component
  Real cy[2][kMaxN];  // y faces (north-face weights)
  Real w[kMaxQ];      // Gauss weights of the rule of this radius
};

// full prediction weights z[R][face][g][m] (face E, W, N, S), for the MOOD
// recompute at any radius, stencil order: b = -R..R, a = -R..R, |a|+|b| <= R
template <class Real>
struct DirectW {
  Real z[4][4][kMaxQ][kMaxN];
  Real w[4][kMaxQ];     // Gauss weights per radius (index 0: FOG, one point)
  Real d2x[5], d2y[5];  // App. B second-derivative weights on the R=1 stencil
  int top;
};

// the cascade of radii: next lower and next higher level of each radius
struct Cascade {
  int next[4];
  int prev[4];
  int top;
};

struct Detect {
  double sigma_v, sigma_p;
  int csd_on;
  double plateau_thr;   // min(dx^3, dy^3)
  double delta;         // min(dx, dy)
  // set by detect_derive: the tests' constants in both precisions, so that
  // no kernel converts or combines them once per cell
  double gm1, hx, hy;   // gamma - 1, 1 / (2 dx), 1 / (2 dy)
  float sigma_v_f, sigma_p_f, plateau_thr_f, delta_f, gm1_f, hx_f, hy_f;
};

// the derived members of D, once its own members and the grid are set
inline void detect_derive(Detect& D, const Grid& g) {
  D.gm1 = g.gamma - 1.0;
  D.hx = 0.5 * g.inv_dx;
  D.hy = 0.5 * g.inv_dy;
  D.sigma_v_f = (float)D.sigma_v;
  D.sigma_p_f = (float)D.sigma_p;
  D.plateau_thr_f = (float)D.plateau_thr;
  D.delta_f = (float)D.delta;
  D.gm1_f = (float)(g.gamma - 1.0);
  D.hx_f = 0.5f * (float)g.inv_dx;
  D.hy_f = 0.5f * (float)g.inv_dy;
}

// one RK stage as buffer roles (slots relative to the step's rotation of
// the state buffers) and the coefficients of StageArgs; w, out2 = -1: none
struct StageSpec {
  int in, out, u0, w, out2;
  double h, ca, cb, wa, wb;
  double tfrac;  // time of the stage input as a fraction of dt
};

struct Scheme {
  int nstages, nbuf, advance;  // stages, state buffers, rotation per step
  StageSpec st[5];
};

template <class Real>
struct StageArgs {
  const double* X;   // ghosted stage input
  const Real* Xr;    // the same in Real: X itself (FP64), its float shadow (FP32)
  const double* U0;  // ghosted U^n (combination)
  double* out;       // ghosted stage output
  Real* outr;        // float shadow of out (FP32), null (FP64)
  double* Fx;        // face-averaged fluxes, FP64 on both paths: each float flux is
  double* Fy;        // widened once, by the face kernel, not once per neighbour
  uint8_t* fbx;      // per x face: bit 0 its left, bit 1 its right state failed the
  uint8_t* fby;      // face-state check (per y face: lower, upper), at the face's radius
  uint8_t* ord;      // radius per cell, this stage
  uint8_t* first;    // first-pass troubled map, this stage
  int* queue;        // troubled cells (first pass output)
  int* qcount;
  const Scalars* sc;
  Scalars* scw;
  int stage;
  // the RK stage as a forward-Euler sub-step and a combination (eqs. rk3,
  // rk4): candidate Y = X - h dt F(X); out = ca U0 + cb Y (ca = 0: U0 unread);
  // with out2 set, also out2 = wa W + wb Y
  double h, ca, cb;
  const double* W;
  double* out2;
  double wa, wb;
};

// the two queues alternate: one holds the cells of the current iteration,
// the other receives the cells troubled in it.  The cells of the queue
// worked on with stamp value v carry v in stamp array v % 2 (two arrays of
// stamp_stride entries each).
struct MoodArgs {
  int* queue[2];
  uint32_t* stamp;
  long long stamp_stride;
  Scalars* sc;
};

// state adjoints of the faces, [v][g][face]; faces of one direction
struct AdjFaces {
  void* L;        // Real, state adjoints of the left/lower cell
  void* R;        // Real, of the right/upper cell
  uint8_t* K;     // EDP1 radius per face
  long long nf;   // faces of this direction
};

// one problem of a batch: its grid, detection constants, second-derivative
// weights (physical units, so per grid) and its place in the pooled buffers
struct Prob {
  Grid g;
  Detect det;
  double d2x[5], d2y[5];
  float d2xf[5], d2yf[5];
  long long state_off;  // elements into each pooled ghosted state
  long long fx_off, fy_off;
  int cell_off;         // cells into the pooled per-cell arrays
  int ncell;
};

// work item of a persistent batched kernel: problem and block coordinates
struct Item {
  int p, a, b, pad;
};

}  // namespace gpm
