// FP32 instantiation of the half-stage kernels and their launchers.
#include "launch_impl.cuh"

namespace spstd {
template struct Launch<float>;
}
