// FP32 instantiation of the half-stage kernels and their launchers.
#include "launch_impl.cuh"
#include "pass_tma.cuh"
#include "pass_tma_launch.h"

namespace spstd {
template struct Launch<float>;

namespace {

// Persistent grid size per (kernel, device): SMs x resident blocks per SM.
template <auto Kernel>
cudaError_t persistent_grid(int threads, size_t smem, int *grid)
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

// Complex points per thread of the pipelined x and strided passes.
template <int N>
constexpr int tma_e_x()
{
    return 16;
}
template <int N>
constexpr int tma_e_s()
{
    return 16;
}

template <int N>
cudaError_t pass_n(int axis, const CUtensorMap *ms, const CUtensorMap *md, const TmaPassArgs *a, cudaStream_t s)
{
    constexpr size_t smem = tma_pass_smem<N>();
    int grid = 0;
    cudaError_t e;
    if (axis == 0) {
        constexpr int E = tma_e_x<N>(), TT = N / E;
        e = persistent_grid<xpass_tma_kernel<N, E>>(16 * TT, smem, &grid);
        if (e != cudaSuccess || !a) return e;
        if (a->n_tiles < grid) grid = a->n_tiles;
        if (grid <= 0) return cudaSuccess;
        xpass_tma_kernel<N, E><<<grid, dim3(TT, 16), smem, s>>>(*ms, *md, *a);
    } else {
        constexpr int E = tma_e_s<N>(), TT = N / E;
        e = persistent_grid<spass_tma_kernel<N, E>>(16 * TT, smem, &grid);
        if (e != cudaSuccess || !a) return e;
        if (a->n_tiles < grid) grid = a->n_tiles;
        if (grid <= 0) return cudaSuccess;
        spass_tma_kernel<N, E><<<grid, dim3(16, TT), smem, s>>>(*ms, *md, *a);
    }
    return cudaGetLastError();
}

cudaError_t pass_any(int axis, int N, const CUtensorMap *ms, const CUtensorMap *md, const TmaPassArgs *a,
                     cudaStream_t s)
{
    switch (N) {
    case 64: return pass_n<64>(axis, ms, md, a, s);
    case 128: return pass_n<128>(axis, ms, md, a, s);
    case 256: return pass_n<256>(axis, ms, md, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_pass_tma(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s)
{
    return pass_any(axis, N, &msrc, &mdst, &a, s);
}

cudaError_t prepare_pass_tma(int axis, int N) { return pass_any(axis, N, nullptr, nullptr, nullptr, nullptr); }
}
