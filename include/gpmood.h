/*
 * gpmood.h -- C ABI of the GB300 GP-MOOD hot path.
 *
 * The method is GP-MOOD (Bourgeois & Lee, arXiv:2110.08683): finite-volume
 * updates of the 2D Euler equations (Sec. 2.1, eqs. gov, euler_eqn,
 * fvm_discrete, fvm_F) with Gaussian-process face reconstruction of radius R
 * and order 2R+1 (Sec. 2.2-2.5, eqs. SE-pred, SE-cov, gp_reconstructor,
 * normalized_z), HLLC fluxes at Gauss points (Table QR), SSP-RK3 (Sec. 3.8,
 * eq. rk3) and the a-posteriori MOOD loop (Sec. 3, Sec. 4 Steps 1-10: CAD,
 * PAD, CSD, plateau, DMP, u2, EDP1 face orders, cascade to first-order
 * Godunov).
 *
 * Conventions for every call:
 *  - Return 0 (GPMOOD_OK) on success or a negative GPMOOD_E_* code.  No
 *    exception or signal crosses the ABI.  After a numerical error
 *    (GPMOOD_E_MOOD_CAP, GPMOOD_E_DT) the handle stays valid so that the state
 *    can be read back.
 *  - A handle owns all of its device memory (cudaMalloc at create, freed at
 *    destroy).  Pointers passed in are borrowed for the duration of the call.
 *  - Work is ordered on the handle's CUDA stream (the legacy default stream
 *    unless gpmood_set_stream gave another).  Calls that return host data
 *    synchronise that stream; gpmood_step_async returns without waiting and
 *    every later call that reads the state, the time or the flags waits for
 *    the queued steps first.
 *  - Also in the ABI: HLL fluxes (Sec. 5.3), the five-stage SSP-RK4 (eq. rk4),
 *    POL-MOOD3 (Sec. 3.1 (iv)), the 1D method, the reverse mode of the step,
 *    batches of independent problems and an allocation-free step.
 *  - State arrays are conservative cell averages U = (rho, rho u, rho v, rho E)
 *    in double precision, structure-of-arrays: U[v*ny*nx + j*nx + i] for
 *    variable v < 4, row j < ny, column i < nx (no ghost cells).
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef GPMOOD_H
#define GPMOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpmood_s* gpmood_t;

/* boundary kinds per side, sides ordered W, E, S, N */
enum {
  GPMOOD_BC_PERIODIC = 0,   /* both sides of an axis must be periodic */
  GPMOOD_BC_OUTFLOW = 1,    /* zero gradient: ghosts copy the nearest interior cell */
  GPMOOD_BC_REFLECT = 2,    /* mirror, normal momentum negated */
  GPMOOD_BC_DIRICHLET = 3,  /* fixed primitive state bc_prim[side] */
  GPMOOD_BC_DMR_BOTTOM = 4, /* S only: x < dmr_wall_x0 -> dmr_post, else reflect */
  GPMOOD_BC_DMR_TOP = 5,    /* N only: x < dmr_xs0 + dmr_xs_speed t -> dmr_post, else dmr_pre */
  GPMOOD_BC_JET = 6         /* S or N: jet_prim[side] for ghost-cell centres with
                               jet_x0 <= x <= jet_x1, outflow elsewhere (Sec. 5.3, the Mach jets) */
};

enum { GPMOOD_FP64 = 0, GPMOOD_FP32 = 1 };

enum {
  GPMOOD_OK = 0,
  GPMOOD_E_INVAL = -1,     /* bad argument */
  GPMOOD_E_CUDA = -2,      /* a CUDA call failed */
  GPMOOD_E_OOM = -3,       /* device allocation failed */
  GPMOOD_E_WEIGHTS = -4,   /* covariance matrix not positive definite in the weight solve */
  GPMOOD_E_MOOD_CAP = -5,  /* the MOOD loop reached max_mood_iters with cells still flagged */
  GPMOOD_E_DT = -6,        /* the time step came out non-positive or not finite */
  GPMOOD_E_NOSTATE = -7,   /* step/run/get before set_state */
  GPMOOD_E_TOO_BIG = -8,   /* grid needs more than the static scratch of gpmood_step_noalloc */
  GPMOOD_E_SYNC = -9       /* a grid-wide barrier of the MOOD loop kernel waited more than
                              about a second (its blocks were not all resident); the step
                              failed and the state is as before it */
};

/* grid and boundary description (Sec. 2.1); caller-owned, copied at create */
typedef struct {
  int nx, ny;                 /* interior cells, each >= max(R_max + 1, 3) (ny = 1 in 1D) */
  double x0, x1, y0, y1;      /* domain; dx = (x1-x0)/nx, dy = (y1-y0)/ny */
  int bc[4];                  /* GPMOOD_BC_* for W, E, S, N */
  double bc_prim[4][4];       /* (rho, u, v, p) for DIRICHLET sides */
  double dmr_post[4], dmr_pre[4];            /* primitive states for the DMR kinds */
  double dmr_wall_x0, dmr_xs0, dmr_xs_speed; /* DMR wall start and shock line x_s(t) */
  double jet_x0, jet_x1;      /* inflow slit of GPMOOD_BC_JET */
  double jet_prim[2][4];      /* jet (rho, u, v, p) on the S and N sides */
  int dim;                    /* 0 or 2: two-dimensional.  1: one-dimensional (ny = 1; y0, y1
                                 and the S/N boundaries are ignored): the stencil a = -R..R,
                                 one point per face, x faces only, detection and the time
                                 step on the x terms alone.  Single-problem handles only */
} gpmood_grid;

/* options; a zero-initialised struct (or NULL) gives the paper's defaults */
typedef struct {
  int ncascade;         /* 0: the full cascade R_max, R_max-1, ..., 1, 0 */
  int cascade[4];       /* GP radii, strictly decreasing, ending with 0 (FOG), e.g. {3,1,0} */
  int precision;        /* GPMOOD_FP64 (default) or GPMOOD_FP32 (reconstruction, Riemann
                           solver and detection in FP32; state and stage sums in FP64) */
  double sigma_v;       /* CSD threshold on -div V (0 -> 5, Sec. 3.4) */
  double sigma_p;       /* CSD threshold on the normalised |grad p| (0 -> 5) */
  int csd_off;          /* 1 disables CSD (Step 6) */
  int max_mood_iters;   /* cap on MOOD iterations per RK stage (0 -> 64 + 4 max(nx, ny)) */
  int riemann;          /* 0: HLLC (Toro et al. 1994, the default); 1: HLL (Harten, Lax, van
                           Leer 1983, the paper's choice for the Mach jets); the same wave
                           speeds.  The adjoint requires HLLC */
  int rk;               /* 0 or 3: SSP-RK3 (eq. rk3).  4: the five-stage SSP-RK4 (eq. rk4), its
                           Dt F(U^(3)) term of the final combination read with a minus
                           sign; each stage's MOOD candidate is its forward-Euler
                           sub-step.  Single-problem handles, no adjoint */
  int eager;            /* 0: one captured CUDA graph per step (no host round trip in a
                           step); 1: every kernel launched on the stream and the host
                           reading the step's counters after each stage.  Either way the
                           MOOD loop of a stage is one cooperative kernel that iterates on
                           the device.  Same kernels, same results; eager is slower, but
                           visible kernel by kernel to profilers that cannot look inside
                           graphs with conditional nodes */
  int recon;            /* 0: GP reconstruction (GP-MOOD).  1: POL-MOOD3 (Sec. 3.1 (iv)):
                           the R = 1 rung is Poly3, the quadratic of eq. poly3 fitted to
                           the five cell averages of the R = 1 stencil (eq. p3_coeffs),
                           at the same Gauss points; the u2 curvatures are Poly3's
                           second derivatives (the centred differences); ell is unused.
                           Requires R_max = 1 (the cascade Poly3 -> FOG).  Single-problem
                           handles and gpmood_step_noalloc */
  int serial_launch;    /* 0: the kernels of a step are launched with programmatic
                           dependent launch (each is scheduled while its predecessor
                           drains and waits for it before touching memory); 1: plain
                           stream order.  Same results */
  int split_faces;      /* 0: on two-dimensional grids one kernel solves the x and the y
                           faces of the first pass, every cell forming its stencil sums
                           once for both; 1: one kernel per direction.  Same results,
                           bit for bit */
} gpmood_options;

/* per-step diagnostics of the most recent step */
typedef struct {
  double t;             /* simulation time after the step */
  double dt;            /* the step's Delta t */
  long long nsteps;     /* steps taken since set_state */
  int iters[5];         /* MOOD iterations per RK stage (3 stages SSP-RK3, 5 SSP-RK4) */
  int nbad_first[5];    /* troubled cells after the first pass, per stage */
  int nbad_total[5];    /* troubled cells summed over all iterations, per stage */
  int nfog_pad[5];      /* FOG candidates failing PAD (accepted per Step 10, reported) */
  int status;           /* GPMOOD_OK or the error code of the last step */
} gpmood_stats;

/*
 * Create a handle for one grid.  gamma: ratio of specific heats; R_max in
 * 0..3 is the top GP radius (0 = FOG only); ell the SE length scale in
 * physical units (ell = 12 dx in most of the paper's runs).  Solves the GP
 * prediction vectors for every radius of the cascade in binary128 (Sec. 2.5),
 * stores them in double and float, and allocates the device buffers.
 * Returns GPMOOD_E_INVAL for bad sizes/kinds, GPMOOD_E_WEIGHTS if a
 * covariance matrix is not positive definite, GPMOOD_E_OOM / _CUDA on
 * allocation failures.  *out is NULL on failure.
 */
int gpmood_create(const gpmood_grid* grid, double gamma, int R_max, double ell,
                  const gpmood_options* opts, gpmood_t* out);

/* Use this CUDA stream (a cudaStream_t, may be NULL for the legacy stream). */
int gpmood_set_stream(gpmood_t h, void* stream);

/* Copy the cell averages U (layout above) in; on_device != 0 means U is a
   device pointer.  Resets t and the step count to 0. */
int gpmood_set_state(gpmood_t h, const double* U, int on_device);

/* Set the simulation time of the current state (time-dependent boundaries
   read it); set_state resets it to 0.  Use it to resume from a checkpoint. */
int gpmood_set_time(gpmood_t h, double t);

/* Copy the current cell averages out (device pointer if on_device != 0). */
int gpmood_get_state(gpmood_t h, double* U, int on_device);

/*
 * One SSP-RK3 step with the MOOD loop in every stage.  Delta t is
 * cfl * min over cells of min(dx/(|u|+c), dy/(|v|+c)), computed on the device
 * (cfl > 0).  If dt_out is non-NULL the call waits and returns Delta t there.
 * Returns GPMOOD_E_MOOD_CAP / GPMOOD_E_DT on numerical failure.
 */
int gpmood_step(gpmood_t h, double cfl, double* dt_out);

/* The same with a given Delta t (> 0) instead of the CFL rule. */
int gpmood_step_dt(gpmood_t h, double dt);

/* Step until t_end, clipping the last step; the step count goes to nsteps_out.
   Graph handles queue the steps in chunks and wait once per chunk; steps
   queued past t_end do nothing (see gpmood_step_async). */
int gpmood_run(gpmood_t h, double t_end, double cfl, long long* nsteps_out);

/*
 * Queue one step like gpmood_step(h, cfl, NULL) on the handle's stream and
 * return without waiting for it or reading anything back.  Each captured
 * step graph opens with a gate: once a step has failed (GPMOOD_E_DT,
 * GPMOOD_E_MOOD_CAP) the queued steps after it do nothing, so the steps
 * that ran are always a prefix of those queued.  The failure is reported by
 * the next gpmood_sync (or gpmood_step / gpmood_run); a failed step leaves
 * the time and the step count where they were.  Every call that reads the
 * state, the time or the flags waits for the queued steps first.  Eager and
 * profiled handles step synchronously here.
 */
int gpmood_step_async(gpmood_t h, double cfl);

/* Wait for the queued steps; GPMOOD_OK or the latched step error. */
int gpmood_sync(gpmood_t h);

/* Kernels launched by the handle's steps since the state was set, counted
   on the device (queued steps included, after waiting for them). */
int gpmood_launch_count(gpmood_t h, long long* count);

/*
 * Diagnostics of the last step (waits).  order_out (nullable, host) receives
 * the final GP radius of every cell in each of the three stages,
 * [3][ny][nx] uint8 (0 = FOG).  first_out (nullable, host) the first-pass
 * troubled-cell map [3][ny][nx] (1 = flagged).  stats_out (nullable).
 */
int gpmood_flags(gpmood_t h, uint8_t* order_out, uint8_t* first_out, gpmood_stats* stats_out);

/* Release the handle and its device memory.  NULL is accepted. */
int gpmood_destroy(gpmood_t h);

/* Static string for a GPMOOD_E_* code. */
const char* gpmood_strerror(int code);

/*
 * Kernel launch count of the last step (device kernels this library
 * launched), for accounting.
 */
int gpmood_last_launches(gpmood_t h);

/* kernel classes for gpmood_kernel_times */
enum {
  GPMOOD_K_DT = 0,      /* time-step reduction */
  GPMOOD_K_GHOST = 1,   /* ghost-cell fill */
  GPMOOD_K_FACES_X = 2, /* first-pass x faces: reconstruction, face CAD, HLLC */
  GPMOOD_K_FACES_Y = 3, /* first-pass y faces */
  GPMOOD_K_UPDATE = 4,  /* first-pass candidate, detection, RK sum, compaction */
  GPMOOD_K_MOOD = 5,    /* MOOD iterations (lower, faces, update) */
  GPMOOD_NKCLASS = 6
};

/*
 * Device-time accounting per kernel class with CUDA events recorded on the
 * handle's stream around every launch.  enable != 0 starts (and zeroes) the
 * accounting, 0 stops it.  Off by default; it adds event records between
 * launches but no synchronisation.
 */
int gpmood_profile(gpmood_t h, int enable);

/* Accumulated milliseconds and launch counts per class (arrays of
   GPMOOD_NKCLASS entries, either may be NULL); waits for the stream. */
int gpmood_kernel_times(gpmood_t h, double* ms, long long* launches);

/*
 * Reverse mode (adjoint) of the step.  The paper defines only the forward
 * scheme; these calls differentiate that scheme (eqs. fvm_discrete, fvm_F,
 * gp_reconstructor, HLLC, rk3) with the GP radius of every cell in every
 * stage and the time step held at the values the forward step chose (the
 * MOOD decisions are not differentiable; holding them is the "frozen mask").
 *
 * gpmood_step_record: one step like gpmood_step (cfl > 0) or gpmood_step_dt
 *   (cfl <= 0 and dt_fixed > 0) that also writes, to caller-owned device
 *   memory, the tape its adjoint needs: tape [3][4][ny][nx] doubles = the
 *   three stage inputs (U^n, U^(1), hat U^(2)), otape [3][ny][nx] bytes = the
 *   final radius of every cell in each stage.  dt_out (nullable, host) gets
 *   the step.
 * gpmood_step_frozen: one step from the current state with the radii of
 *   otape and the given dt, without detection (replays a recorded step; used
 *   for finite differences of the frozen-mask map).
 * gpmood_step_adjoint: lam_out = (dU^{n+1}/dU^n)^T lam_in for the recorded
 *   step (tape, otape, dt, and t its start time), all device arrays in the
 *   state layout; lam_out may not alias lam_in.  Allocates its work buffers
 *   on the first call and waits for the stream.  Where a reconstructed state
 *   has non-positive pressure the Riemann solver's branch is decided by NaN
 *   comparisons; the adjoint follows the branch the forward took.
 * gpmood_step_record_states / gpmood_step_adjoint_states: the same with a
 *   state tape (caller-owned device memory of gpmood_state_tape_bytes bytes
 *   per step): the recorded step also keeps the reconstructed states every
 *   final face flux was solved from (eq. gp_reconstructor at the face's EDP1
 *   radius, the Gauss points of Table QR), and the adjoint reads them instead
 *   of reconstructing them again.  Two-dimensional grids.  The gradient is the
 *   same, bit for bit; the state tape spends device memory (8 q N_faces reals
 *   a stage, q the top radius's rule) to save the reconstruction's arithmetic.
 */
int gpmood_step_record(gpmood_t h, double cfl, double dt_fixed, double* tape, uint8_t* otape,
                       double* dt_out);
int gpmood_step_frozen(gpmood_t h, const uint8_t* otape, double dt);
int gpmood_step_adjoint(gpmood_t h, const double* tape, const uint8_t* otape, double dt, double t,
                        const double* lam_in, double* lam_out);
int gpmood_state_tape_bytes(gpmood_t h, size_t* bytes);
int gpmood_step_record_states(gpmood_t h, double cfl, double dt_fixed, double* tape,
                              uint8_t* otape, void* stape, double* dt_out);
int gpmood_step_adjoint_states(gpmood_t h, const double* tape, const uint8_t* otape,
                               const void* stape, double dt, double t, const double* lam_in,
                               double* lam_out);

/*
 * Batches: many independent problems of uneven sizes advanced together.
 * Every problem has its own grid and boundaries and its own time step; all
 * share gamma, R_max, the cascade and the options, and the GP weights, so
 * ell/dx and ell/dy must be the same for every problem (ell = c * dx with
 * one c, as in ell = 12 dx).  Each kernel class runs as one persistent
 * launch that walks (problem, block) work items; a step is one captured
 * graph whose MOOD loops run on the device.  The first step times the face
 * kernel variants (4 or 8 warps, i.e. rows or columns, per work item) and
 * keeps the faster per sweep.
 *
 * State arrays of a batch are the problems' arrays (layout above) one after
 * the other, in problem order.  Errors as for the single-problem calls; the
 * MOOD iteration cap applies to the whole batch.
 */
typedef struct gpmood_batch_s* gpmood_batch_t;

/* grids[nprob], ell[nprob]: per problem; the other arguments as for
   gpmood_create.  GPMOOD_E_INVAL if the problems need different weights. */
int gpmood_batch_create(const gpmood_grid* grids, int nprob, double gamma, int R_max,
                        const double* ell, const gpmood_options* opts, gpmood_batch_t* out);
int gpmood_batch_set_stream(gpmood_batch_t b, void* stream);
/* all problems' cell averages, concatenated; resets every problem's time */
int gpmood_batch_set_state(gpmood_batch_t b, const double* U, int on_device);
int gpmood_batch_get_state(gpmood_batch_t b, double* U, int on_device);
/* one SSP-RK3 step of every problem with its own CFL time step (waits) */
int gpmood_batch_step(gpmood_batch_t b, double cfl);
/* step until every problem has reached t_end (each clips its last step);
   nsteps_out gets the number of batch steps */
int gpmood_batch_run(gpmood_batch_t b, double t_end, double cfl, long long* nsteps_out);
/* per-problem time, last step and step count (arrays of nprob, nullable);
   total (nullable) gets the summed MOOD statistics of the last step */
int gpmood_batch_info(gpmood_batch_t b, double* t, double* dt, long long* nsteps,
                      gpmood_stats* total);
/* the autotuner's choice of first-pass face kernel, made on the first step:
   per sweep (x, y) the warps per block (4 or 8) and the number of work items
   (blocks), or warps = {0, 0} for the kernel that solves both directions,
   blocks then its work items; GPMOOD_E_NOSTATE before the first step */
int gpmood_batch_tuning(gpmood_batch_t b, int* warps, int* blocks);
/* the update kernel's tuned grid (blocks walking the update items) and the
   grid of the MOOD loop kernel (co-resident blocks); GPMOOD_E_NOSTATE before
   the first step */
int gpmood_batch_grids(gpmood_batch_t b, int* update_blocks, int* mood_blocks);
int gpmood_batch_profile(gpmood_batch_t b, int enable);
int gpmood_batch_kernel_times(gpmood_batch_t b, double* ms, long long* launches);
int gpmood_batch_destroy(gpmood_batch_t b);

/*
 * gpmood_step_noalloc -- one SSP-RK3 step with the MOOD loop that allocates
 * no memory at all.  The paper has no counterpart; this is a service for
 * callers that cannot allocate device memory while they run, for example a
 * host framework that owns the whole device memory pool and forbids raw
 * cudaMalloc/cudaFree (both synchronise the device and fragment the pool),
 * or a real-time loop that must not allocate after start-up.
 *
 * The step runs the same kernels as gpmood_step on a temporary handle whose
 * buffers (three ghosted states, face fluxes, flag maps, queues, counters)
 * are carved out of one file-scope device array of
 * GPMOOD_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads this
 * library holds until the process exits.  At R_max = 3 that covers square
 * grids up to 292 x 292 cells in FP64 and 256 x 256 in FP32 (whose float
 * shadows of the three states share the array); a grid needing more returns
 * GPMOOD_E_TOO_BIG without touching the device.
 *
 * Arguments are those of gpmood_create (grid, gamma, R_max, ell, opts),
 * checked as it checks them, except that only SSP-RK3 (opts->rk 0 or 3) and
 * two-dimensional grids (grid->dim 0 or 2) are taken; anything else returns
 * GPMOOD_E_INVAL before the device is touched.  In addition:
 * U_in / U_out, device pointers to cell averages in the layout above (they
 * may be the same array); t, the time of U_in (time-dependent boundaries);
 * cfl > 0; dt_out (nullable, host) receives the step's Delta t; stream, a
 * cudaStream_t or NULL.  The call waits for the stream before it returns.
 *
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress with that device current); make that first
 * call before any stream capture.  Every call shares the one array and
 * leaves its contents behind; the parts that must start at zero are cleared
 * at each call.  Calls that overlap on the same GPU (other threads or
 * streams) race on its scratch, so serialise them.  Each GPU has its own
 * array, and the host-side copy of the step's counters lives on the
 * caller's stack, so calls on different GPUs share nothing.  Errors as for
 * gpmood_step.
 */
#define GPMOOD_NOALLOC_SCRATCH_BYTES (16u << 20)
int gpmood_step_noalloc(const gpmood_grid* grid, double gamma, int R_max, double ell,
                        const gpmood_options* opts, const double* U_in, double* U_out, double t,
                        double cfl, double* dt_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
