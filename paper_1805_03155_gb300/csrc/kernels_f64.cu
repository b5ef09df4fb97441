// FP64 instantiation of the half-stage kernels and their launchers.
#include "launch_impl.cuh"

namespace spstd {
template struct Launch<double>;

__global__ void sum_partials_kernel(const double *__restrict__ partial, int count, double *__restrict__ out)
{
    __shared__ double s_w[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc, s_w);
    if (threadIdx.x == 0) *out = acc;
}

cudaError_t launch_sum_partials(const double *partial, int count, double *out, cudaStream_t s)
{
    sum_partials_kernel<<<1, 256, 0, s>>>(partial, count, out);
    return cudaGetLastError();
}
}
