// persist.cuh -- grid size of a persistent kernel: SMs x resident blocks per SM.
#pragma once

#include <cuda_runtime.h>

namespace spstd {

// Persistent grid size per (kernel, device): SMs x resident blocks per SM.
template <auto Kernel>
inline cudaError_t persistent_grid(int threads, size_t smem, int *grid)
{
    static int cached[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!cached[dev]) {
        e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, Kernel, threads, smem);
        if (e != cudaSuccess) return e;
        if (per < 1) return cudaErrorInvalidConfiguration;
        cached[dev] = sms * per;
    }
    *grid = cached[dev];
    return cudaSuccess;
}

}  // namespace spstd
