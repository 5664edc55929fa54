// gpmood_launch.h -- host-side launchers of the precision-templated kernels.
#pragma once

#include "gpmood_internal.h"

namespace gpm {

// programmatic dependent launch between the kernels of a step: the next
// kernel is scheduled while its predecessor drains and waits in
// griddepcontrol.wait (pdl_wait, its first statement) until the predecessor
// has completed and its writes are visible.  Set per thread by the API
// around a capture or an eager step.
extern thread_local int g_pdl;

// the same with dynamic shared memory
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ks(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                            Args... args) {
  return launch_ks(kernel, grid, block, 0, st, args...);
}

template <class Real>
struct Launch {
  // first pass: x (dir 0) or y (dir 1) faces at the top radius
  static cudaError_t faces(int top, int dir, const StageArgs<Real>& A, const Grid& g,
                           const ParityW<Real>& W, cudaStream_t st);
  // first pass: x and y faces in one launch (two-dimensional grids)
  static cudaError_t faces_xy(int top, const StageArgs<Real>& A, const Grid& g,
                              const ParityW<Real>& W, cudaStream_t st);
  // once per process and device: kernel attributes (shared-memory limits)
  static cudaError_t prepare();
  static cudaError_t update_first(const StageArgs<Real>& A, const Grid& g, const Detect& D,
                                  const DirectW<Real>& Wd, cudaStream_t st);
  // the whole MOOD loop of stage `stage` in one launch of `blocks` co-resident
  // blocks (cooperative when `coop`)
  static cudaError_t mood_loop(const StageArgs<Real>& A, const MoodArgs& M, const Grid& g,
                               const Detect& D, const DirectW<Real>& Wd, const Cascade& C,
                               int stage, const LoopTail& T, int blocks, int coop,
                               cudaStream_t st);
  // co-resident blocks of the MOOD loop kernel on this device (its grid)
  static int mood_loop_blocks();
};

// replay with given radii, and the reverse-mode passes of the adjoint
template <class Real>
struct LaunchA {
  static cudaError_t frozen_stage(const StageArgs<Real>& A, const Grid& g,
                                  const DirectW<Real>& Wd, cudaStream_t st);
  // X: the ghosted stage input in Real (converted into Xr when Real is float)
  static cudaError_t adj_faces(const double* X, void* Xr, const double* v, const uint8_t* ord,
                               const Grid& g, const ParityW<Real>& W, const DirectW<Real>& Wd,
                               const AdjFaces& Ax, const AdjFaces& Ay, cudaStream_t st);
  // pass 1 from a recorded step's state tape st (of this stage)
  static cudaError_t adj_faces_stored(const void* st, const double* v, const uint8_t* ord,
                                      const Grid& g, const ParityW<Real>& W,
                                      const DirectW<Real>& Wd, const AdjFaces& Ax,
                                      const AdjFaces& Ay, cudaStream_t st_);
  static cudaError_t adj_gather(const Grid& g, const DirectW<Real>& Wd, const AdjFaces& Ax,
                                const AdjFaces& Ay, double* G, cudaStream_t st);
};

// batched launchers: persistent grids walking work-item lists
template <class Real>
struct LaunchB {
  static cudaError_t faces(int top, int dir, int fw, const StageArgs<Real>& B, const Prob* probs,
                           const Scalars* psc, const Item* items, int nitems, int blocks,
                           const ParityW<Real>& W, cudaStream_t st);
  // max resident blocks per SM of a face kernel variant
  static int faces_occupancy(int top, int dir, int fw);
  // both directions in one kernel over (problem, segment, band) items
  static cudaError_t faces_xy(int top, const StageArgs<Real>& B, const Prob* probs,
                              const Scalars* psc, const Item* items, int nitems,
                              const ParityW<Real>& W, cudaStream_t st);
  static cudaError_t prepare();
  static cudaError_t update(const StageArgs<Real>& B, const Prob* probs, const Scalars* psc,
                            const Item* items, int nitems, int blocks, const DirectW<Real>& Wd,
                            cudaStream_t st);
  // the MOOD loop of stage `stage` of every problem in one launch of
  // `blocks` co-resident blocks (cooperative when `coop`)
  static cudaError_t mood_loop(const StageArgs<Real>& B, const MoodArgs& M, const Prob* probs,
                               const Scalars* psc, int nprob, const DirectW<Real>& Wd,
                               const Cascade& C, int stage, int blocks, int coop,
                               cudaStream_t st);
  static int mood_loop_blocks();
};

// Xf: float shadow of X (FP32 path) or null
cudaError_t launch_fill(double* X, float* Xf, const Grid& g, const Scalars* sc, double tfrac,
                        cudaStream_t st);
// Xf: float shadow of X (FP32 path: the CFL rate in float) or null
cudaError_t launch_dt(const double* X, const float* Xf, const Grid& g, Scalars* sc, cudaStream_t st);
cudaError_t launch_finish(Scalars* sc, int base, cudaStream_t st);
cudaError_t launch_gate(Scalars* sc, cudaGraphConditionalHandle hif, cudaStream_t st);

}  // namespace gpm
