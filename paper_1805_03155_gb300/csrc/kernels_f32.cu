// FP32 instantiation of the half-stage kernels and their launchers.
#include "launch_impl.cuh"
#include "pass_tma.cuh"
#include "pass_tma_launch.h"
#include "pass_xy.cuh"
#include "persist.cuh"

namespace spstd {
template struct Launch<float>;

namespace {

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

template <int N>
cudaError_t xy_n(const CUtensorMap *maps, const XyPassArgs *a, cudaStream_t s)
{
    constexpr int E = 16, TT = N / E;
    constexpr int threads = 16 * TT + 32;  // compute warps + the producer warp
    constexpr size_t smem = xy_pass_smem<N>();
    int grid = 0;
    cudaError_t e = persistent_grid<xypass_tma_kernel<N, E>>(threads, smem, &grid);
    if (e != cudaSuccess || !a) return e;
    // lag: the list keeps each plane's x tiles about four grids' worth of items
    // behind its y tiles, so that the plane is normally finished when they are claimed
    XyPassArgs b = *a;
    const int per_plane = b.nxt + b.nyt;
    b.lag = per_plane > 0 ? (4 * grid + per_plane - 1) / per_plane : 1;
    xypass_tma_kernel<N, E><<<grid, threads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], b);
    return cudaGetLastError();
}

cudaError_t xy_any(int N, const CUtensorMap *maps, const XyPassArgs *a, cudaStream_t s)
{
    switch (N) {
    case 64: return xy_n<64>(maps, a, s);
    case 128: return xy_n<128>(maps, a, s);
    case 256: return xy_n<256>(maps, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_xypass_tma(int N, const CUtensorMap &src_x, const CUtensorMap &dst_x, const CUtensorMap &src_y,
                              const CUtensorMap &dst_y, const XyPassArgs &a, cudaStream_t s)
{
    const CUtensorMap maps[4] = {src_x, dst_x, src_y, dst_y};
    return xy_any(N, maps, &a, s);
}

cudaError_t prepare_xypass_tma(int N) { return xy_any(N, nullptr, nullptr, nullptr); }

cudaError_t launch_pass_tma(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s)
{
    return pass_any(axis, N, &msrc, &mdst, &a, s);
}

cudaError_t prepare_pass_tma(int axis, int N) { return pass_any(axis, N, nullptr, nullptr, nullptr, nullptr); }
}
