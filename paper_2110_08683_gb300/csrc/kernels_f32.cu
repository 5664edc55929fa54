// kernels_f32.cu -- FP32 instantiation: reconstruction, Riemann solver and
// detection in float; state, candidate and RK sums in double.
#include "kernels_impl.cuh"
template struct gpm::Launch<float>;
template struct gpm::LaunchB<float>;
template struct gpm::LaunchA<float>;
