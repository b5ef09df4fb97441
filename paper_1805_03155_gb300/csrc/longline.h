// longline.h -- host entry points of the four-step long-line x pass.
#pragma once

#include <cuda_runtime.h>

#include "longline.cuh"

namespace spstd {

// Largest x line the four-step pass takes (N1 <= 1024 columns of N2 <= 4096).
constexpr int64_t kMaxLongN = int64_t(1) << 22;

// The split N = N1 N2 used for a long line of N points (N a power of two,
// 2048 <= N <= kMaxLongN): N2 = min(4096, N/2).
inline void long_split(int64_t N, int *N1, int *N2)
{
    *N2 = (int)(N / 2 < 4096 ? N / 2 : 4096);
    *N1 = (int)(N / *N2);
}

// dst += L_x-term + bV V src over all lines (three launches on s).
template <typename T>
cudaError_t launch_long_x(const LongArgs<T> &a, cudaStream_t s, int which = -1);

// Raises the shared-memory limits of the three kernels (call outside capture).
template <typename T>
cudaError_t prepare_long_x(int N1, int N2);

}  // namespace spstd
