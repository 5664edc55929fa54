// kernels_impl.cuh -- launcher bodies, instantiated once per precision.
#pragma once

#include "adjoint_kernels.cuh"
#include "gpmood_kernels.cuh"
#include "gpmood_launch.h"

namespace gpm {

template <int R, class Real>
static cudaError_t faces_r(int dir, const StageArgs<Real>& A, const Grid& g,
                           const ParityW<Real>& W, cudaStream_t st) {
  dim3 blk(32, kFaceWarps);
  if (dir == 0) {
    dim3 gx((g.nx + 1 + kSegFaces - 1) / kSegFaces, (g.ny + kFaceWarps - 1) / kFaceWarps);
    return launch_k(k_faces<R, Real, 0, kFaceWarps>, gx, blk, st, A, g, W);
  }
  dim3 gy((g.nx + kFaceWarps - 1) / kFaceWarps, (g.ny + 1 + kSegFaces - 1) / kSegFaces);
  return launch_k(k_faces<R, Real, 1, kFaceWarps>, gy, blk, st, A, g, W);
}

template <class Real>
cudaError_t Launch<Real>::faces(int top, int dir, const StageArgs<Real>& A, const Grid& g,
                                const ParityW<Real>& W, cudaStream_t st) {
  switch (top) {
    case 0: return faces_r<0, Real>(dir, A, g, W, st);
    case 1: return faces_r<1, Real>(dir, A, g, W, st);
    case 2: return faces_r<2, Real>(dir, A, g, W, st);
    default: return faces_r<3, Real>(dir, A, g, W, st);
  }
}

template <int R, class Real>
static cudaError_t faces_xy_r(const StageArgs<Real>& A, const Grid& g, const ParityW<Real>& W,
                              cudaStream_t st) {
  dim3 grd((g.nx + 1 + kSegFaces - 1) / kSegFaces, (g.ny + 1 + kXYBand - 1) / kXYBand);
  return launch_ks(k_faces_xy<R, Real>, grd, dim3(32, kXYRows), sizeof(XYShared<R, Real>), st,
                   A, g, W);
}

template <class Real>
cudaError_t Launch<Real>::faces_xy(int top, const StageArgs<Real>& A, const Grid& g,
                                   const ParityW<Real>& W, cudaStream_t st) {
  switch (top) {
    case 0: return faces_xy_r<0, Real>(A, g, W, st);
    case 1: return faces_xy_r<1, Real>(A, g, W, st);
    case 2: return faces_xy_r<2, Real>(A, g, W, st);
    default: return faces_xy_r<3, Real>(A, g, W, st);
  }
}

template <int R, class Real>
static cudaError_t xy_attr() {
  return cudaFuncSetAttribute(k_faces_xy<R, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(XYShared<R, Real>));
}

template <class Real>
cudaError_t Launch<Real>::prepare() {
  cudaError_t e = xy_attr<0, Real>();
  if (e == cudaSuccess) e = xy_attr<1, Real>();
  if (e == cudaSuccess) e = xy_attr<2, Real>();
  if (e == cudaSuccess) e = xy_attr<3, Real>();
  return e;
}

template <class Real>
cudaError_t Launch<Real>::update_first(const StageArgs<Real>& A, const Grid& g, const Detect& D,
                                       const DirectW<Real>& Wd, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  return launch_k(k_update_first<Real>, grd, blk, st, A, g, D, Wd);
}

template <class Real>
cudaError_t Launch<Real>::mood_loop(const StageArgs<Real>& A, const MoodArgs& M, const Grid& g,
                                    const Detect& D, const DirectW<Real>& Wd, const Cascade& C,
                                    int stage, const LoopTail& T, int blocks, int coop,
                                    cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  // cooperative: the launch fails rather than run a grid whose blocks cannot
  // all be resident at once (the barriers need them all)
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = coop ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_mood_loop<Real>, A, M, g, D, Wd, C, stage, T);
}

template <class Real>
int Launch<Real>::mood_loop_blocks() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mood_loop<Real>, 256, 0) !=
          cudaSuccess || sms <= 0 || occ <= 0) {
    cudaGetLastError();
    return 0;
  }
  // two blocks an SM where they fit: enough warps to hide the FP64 latency
  // of the few cells an iteration works on, few arrivals per barrier
  return sms * (occ < 2 ? occ : 2);
}

template <int R, class Real, int FW>
static cudaError_t faces_batch_r(int dir, const StageArgs<Real>& B, const Prob* probs,
                                 const Scalars* psc, const Item* items, int nitems, int blocks,
                                 const ParityW<Real>& W, cudaStream_t st) {
  dim3 blk(32, FW);
  (void)blocks;  // one block per item
  if (dir == 0) k_faces_batch<R, Real, 0, FW><<<nitems, blk, 0, st>>>(B, probs, psc, items, W);
  else k_faces_batch<R, Real, 1, FW><<<nitems, blk, 0, st>>>(B, probs, psc, items, W);
  return cudaGetLastError();
}

template <int R, class Real>
static cudaError_t faces_batch_fw(int dir, int fw, const StageArgs<Real>& B, const Prob* probs,
                                  const Scalars* psc, const Item* items, int nitems, int blocks,
                                  const ParityW<Real>& W, cudaStream_t st) {
  if (fw == 4) return faces_batch_r<R, Real, 4>(dir, B, probs, psc, items, nitems, blocks, W, st);
  return faces_batch_r<R, Real, 8>(dir, B, probs, psc, items, nitems, blocks, W, st);
}

template <class Real>
cudaError_t LaunchB<Real>::faces(int top, int dir, int fw, const StageArgs<Real>& B,
                                 const Prob* probs, const Scalars* psc, const Item* items,
                                 int nitems, int blocks, const ParityW<Real>& W, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  switch (top) {
    case 0: return faces_batch_fw<0, Real>(dir, fw, B, probs, psc, items, nitems, blocks, W, st);
    case 1: return faces_batch_fw<1, Real>(dir, fw, B, probs, psc, items, nitems, blocks, W, st);
    case 2: return faces_batch_fw<2, Real>(dir, fw, B, probs, psc, items, nitems, blocks, W, st);
    default: return faces_batch_fw<3, Real>(dir, fw, B, probs, psc, items, nitems, blocks, W, st);
  }
}

template <int R, class Real>
static cudaError_t faces_xy_batch_r(const StageArgs<Real>& B, const Prob* probs,
                                    const Scalars* psc, const Item* items, int nitems,
                                    const ParityW<Real>& W, cudaStream_t st) {
  return launch_ks(k_faces_xy_batch<R, Real>, dim3(nitems), dim3(32, kXYRows),
                   sizeof(XYShared<R, Real>), st, B, probs, psc, items, W);
}

template <class Real>
cudaError_t LaunchB<Real>::faces_xy(int top, const StageArgs<Real>& B, const Prob* probs,
                                    const Scalars* psc, const Item* items, int nitems,
                                    const ParityW<Real>& W, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  switch (top) {
    case 0: return faces_xy_batch_r<0, Real>(B, probs, psc, items, nitems, W, st);
    case 1: return faces_xy_batch_r<1, Real>(B, probs, psc, items, nitems, W, st);
    case 2: return faces_xy_batch_r<2, Real>(B, probs, psc, items, nitems, W, st);
    default: return faces_xy_batch_r<3, Real>(B, probs, psc, items, nitems, W, st);
  }
}

template <int R, class Real>
static cudaError_t xy_batch_attr() {
  return cudaFuncSetAttribute(k_faces_xy_batch<R, Real>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(XYShared<R, Real>));
}

template <class Real>
cudaError_t LaunchB<Real>::prepare() {
  cudaError_t e = xy_batch_attr<0, Real>();
  if (e == cudaSuccess) e = xy_batch_attr<1, Real>();
  if (e == cudaSuccess) e = xy_batch_attr<2, Real>();
  if (e == cudaSuccess) e = xy_batch_attr<3, Real>();
  return e;
}

template <int R, class Real>
static int occ_r(int dir, int fw) {
  int n = 0;
  if (fw == 4) {
    if (dir == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_faces_batch<R, Real, 0, 4>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_faces_batch<R, Real, 1, 4>, 128, 0);
  } else {
    if (dir == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_faces_batch<R, Real, 0, 8>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_faces_batch<R, Real, 1, 8>, 256, 0);
  }
  return n > 0 ? n : 1;
}

template <class Real>
int LaunchB<Real>::faces_occupancy(int top, int dir, int fw) {
  switch (top) {
    case 0: return occ_r<0, Real>(dir, fw);
    case 1: return occ_r<1, Real>(dir, fw);
    case 2: return occ_r<2, Real>(dir, fw);
    default: return occ_r<3, Real>(dir, fw);
  }
}

template <class Real>
cudaError_t LaunchB<Real>::update(const StageArgs<Real>& B, const Prob* probs, const Scalars* psc,
                                  const Item* items, int nitems, int blocks,
                                  const DirectW<Real>& Wd, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_update_batch<Real><<<blocks, dim3(32, 8), 0, st>>>(B, probs, psc, items, nitems, Wd);
  return cudaGetLastError();
}

template <class Real>
cudaError_t LaunchB<Real>::mood_loop(const StageArgs<Real>& B, const MoodArgs& M,
                                     const Prob* probs, const Scalars* psc, int nprob,
                                     const DirectW<Real>& Wd, const Cascade& C, int stage,
                                     int blocks, int coop, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = coop ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_mood_loop_batch<Real>, B, M, probs, psc, nprob, Wd, C, stage);
}

template <class Real>
int LaunchB<Real>::mood_loop_blocks() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mood_loop_batch<Real>, 256, 0) !=
          cudaSuccess || sms <= 0 || occ <= 0) {
    cudaGetLastError();
    return 0;
  }
  return sms * (occ < 2 ? occ : 2);
}

template <class Real>
cudaError_t LaunchA<Real>::frozen_stage(const StageArgs<Real>& A, const Grid& g,
                                        const DirectW<Real>& Wd, cudaStream_t st) {
  const long long nfx = (long long)(g.nx + 1) * g.ny, nfy = (long long)g.nx * (g.ny + 1);
  k_faces_frozen<Real, 0><<<(int)((nfx + 127) / 128), 128, 0, st>>>(A, g, Wd);
  k_faces_frozen<Real, 1><<<(int)((nfy + 127) / 128), 128, 0, st>>>(A, g, Wd);
  k_update_frozen<Real><<<dim3((g.nx + 31) / 32, (g.ny + 7) / 8), dim3(32, 8), 0, st>>>(A, g);
  return cudaGetLastError();
}

template <int R, class Real>
static cudaError_t adj_faces_r(const Real* X, const double* v, const uint8_t* ord,
                               const Grid& g, const ParityW<Real>& W, const DirectW<Real>& Wd,
                               const AdjFaces& Ax, const AdjFaces& Ay, cudaStream_t st) {
  // 4 warps a block: the reverse sweep holds ~150-250 registers a thread
  constexpr int FW = 4;
  dim3 blk(32, FW);
  dim3 gx((g.nx + 1 + kSegFaces - 1) / kSegFaces, (g.ny + FW - 1) / FW);
  k_adj_faces_sweep<R, Real, 0, FW><<<gx, blk, 0, st>>>(X, v, ord, g, W, Wd, Ax);
  dim3 gy((g.nx + FW - 1) / FW, (g.ny + 1 + kSegFaces - 1) / kSegFaces);
  k_adj_faces_sweep<R, Real, 1, FW><<<gy, blk, 0, st>>>(X, v, ord, g, W, Wd, Ay);
  return cudaGetLastError();
}

template <class Real>
cudaError_t LaunchA<Real>::adj_faces(const double* X, void* Xr, const double* v,
                                     const uint8_t* ord, const Grid& g, const ParityW<Real>& W,
                                     const DirectW<Real>& Wd, const AdjFaces& Ax,
                                     const AdjFaces& Ay, cudaStream_t st) {
  const Real* XR;
  if (sizeof(Real) == sizeof(double)) {
    XR = (const Real*)X;
  } else {
    k_to_real<Real><<<152 * 8, 256, 0, st>>>(X, (Real*)Xr, 4 * g.vstride);
    XR = (const Real*)Xr;
  }
  switch (Wd.top) {
    case 0: return adj_faces_r<0, Real>(XR, v, ord, g, W, Wd, Ax, Ay, st);
    case 1: return adj_faces_r<1, Real>(XR, v, ord, g, W, Wd, Ax, Ay, st);
    case 2: return adj_faces_r<2, Real>(XR, v, ord, g, W, Wd, Ax, Ay, st);
    default: return adj_faces_r<3, Real>(XR, v, ord, g, W, Wd, Ax, Ay, st);
  }
}

template <class Real>
cudaError_t LaunchA<Real>::adj_faces_stored(const void* st, const double* v, const uint8_t* ord,
                                            const Grid& g, const ParityW<Real>& W,
                                            const DirectW<Real>& Wd, const AdjFaces& Ax,
                                            const AdjFaces& Ay, cudaStream_t s) {
  const int qt = rule_q(Wd.top);
  const Real* t = (const Real*)st;
  const Real* xL = t;
  const Real* xR = t + 4LL * qt * Ax.nf;
  const Real* yL = t + 8LL * qt * Ax.nf;
  const Real* yR = yL + 4LL * qt * Ay.nf;
  k_adj_faces_stored<Real, 0><<<(int)((Ax.nf + 127) / 128), 128, 0, s>>>(xL, xR, qt, v, ord, g,
                                                                         W, Wd, Ax);
  k_adj_faces_stored<Real, 1><<<(int)((Ay.nf + 127) / 128), 128, 0, s>>>(yL, yR, qt, v, ord, g,
                                                                         W, Wd, Ay);
  return cudaGetLastError();
}

template <class Real>
cudaError_t LaunchA<Real>::adj_gather(const Grid& g, const DirectW<Real>& Wd, const AdjFaces& Ax,
                                      const AdjFaces& Ay, double* G, cudaStream_t st) {
  const long long n = (long long)(g.nx + 2 * g.H) * (g.ny + 2 * g.H);
  k_adj_gather<Real><<<(int)((n + 255) / 256), 256, 0, st>>>(g, Wd, Ax, Ay, G);
  return cudaGetLastError();
}

}  // namespace gpm
