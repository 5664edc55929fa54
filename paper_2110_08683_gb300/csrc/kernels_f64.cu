// kernels_f64.cu -- FP64 instantiation of the stage kernels.
#include "kernels_impl.cuh"
template struct gpm::Launch<double>;
template struct gpm::LaunchB<double>;
template struct gpm::LaunchA<double>;
