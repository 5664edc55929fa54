// kernels_impl.cuh -- launcher bodies, instantiated once per precision.
#pragma once

#include "gpmood_kernels.cuh"
#include "gpmood_launch.h"

namespace gpm {

template <int R, class Real>
static cudaError_t faces_r(int dir, const StageArgs<Real>& A, const Grid& g,
                           const ParityW<Real>& W, cudaStream_t st) {
  dim3 blk(32, kFaceWarps);
  if (dir == 0) {
    dim3 gx((g.nx + 1 + kSegFaces - 1) / kSegFaces, (g.ny + kFaceWarps - 1) / kFaceWarps);
    k_faces<R, Real, 0><<<gx, blk, 0, st>>>(A, g, W);
  } else {
    dim3 gy((g.nx + kFaceWarps - 1) / kFaceWarps, (g.ny + 1 + kSegFaces - 1) / kSegFaces);
    k_faces<R, Real, 1><<<gy, blk, 0, st>>>(A, g, W);
  }
  return cudaGetLastError();
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

template <class Real>
cudaError_t Launch<Real>::update_first(const StageArgs<Real>& A, const Grid& g, const Detect& D,
                                       const DirectW<Real>& Wd, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  k_update_first<Real><<<grd, blk, 0, st>>>(A, g, D, Wd);
  return cudaGetLastError();
}

template <class Real>
cudaError_t Launch<Real>::mood_faces(const StageArgs<Real>& A, const MoodArgs& M, const Grid& g,
                                     const DirectW<Real>& Wd, const Cascade& C, cudaStream_t st) {
  k_mood_faces<Real><<<2 * kMoodBlocks, 128, 0, st>>>(A, M, g, Wd, C);
  return cudaGetLastError();
}

template <class Real>
cudaError_t Launch<Real>::mood_update(const StageArgs<Real>& A, const MoodArgs& M, const Grid& g,
                                      const Detect& D, const DirectW<Real>& Wd, cudaStream_t st) {
  k_mood_update<Real><<<kMoodBlocks, 256, 0, st>>>(A, M, g, D, Wd);
  return cudaGetLastError();
}

}  // namespace gpm
