// Instantiations and launchers of the reduce-add pipelined passes
// (pass_tmared.cuh): single grids and batches, lines of 32..512 points.
#include <algorithm>
#include <utility>

#include "pass_tmared.cuh"
#include "persist.cuh"

namespace spstd {
namespace {

// Complex points per thread: tmared_e(N), 16 for power-of-two lines.
// Measured at 256^3: E = 8 (256-thread x blocks, 16 warps per SM) takes
// 0.054 ms per x pass against 0.047 ms for E = 16.

// Launch with programmatic stream serialisation: the kernel may start while
// the previous work on the stream finishes; it waits for it (griddepcontrol)
// after its prologue.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int N, bool BATCH, bool VSEP = false, int EX = tmared_e(N)>
cudaError_t red_x(const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md, const TmaPassArgs *a,
                  const TmaBatchArgs *ba, cudaStream_t s)
{
    using G = XRed<N, EX, BATCH, VSEP>;
    int grid = 0;
    cudaError_t e = persistent_grid<xpass_tmared_kernel<N, EX, BATCH, VSEP>>(G::THREADS, G::SMEM, &grid);
    if (e != cudaSuccess || !(BATCH ? (const void *)ba : (const void *)a)) return e;
    const int total = BATCH ? ba->members * ba->tiles : a->n_tiles;
    if (total < grid) grid = total;
    if (grid <= 0) return cudaSuccess;
    const CUtensorMap none{};
    const TmaPassArgs a0{};
    const TmaBatchArgs b0{};
    return launch_pdl(xpass_tmared_kernel<N, EX, BATCH, VSEP>, dim3(grid), dim3(G::TT, G::LP), G::SMEM, s,
                      BATCH ? none : *ms, BATCH ? none : *mv, BATCH ? none : *md, BATCH ? a0 : *a, BATCH ? *ba : b0);
}

template <int N, bool VSEP, bool BATCH>
cudaError_t red_xw(const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md, const TmaPassArgs *a,
                   const TmaBatchArgs *ba, cudaStream_t s)
{
    using G = XWarp<N, VSEP, BATCH>;
    int grid = 0;
    cudaError_t e = persistent_grid<xpass_warp_kernel<N, VSEP, BATCH>>(G::THREADS, G::SMEM, &grid);
    if (e != cudaSuccess || !(BATCH ? (const void *)ba : (const void *)a)) return e;
    const int total = BATCH ? ba->members * ba->tiles : a->n_tiles;
    const int need = (total + G::WARPS - 1) / G::WARPS;  // blocks that get a tile
    if (need < grid) grid = need;
    if (grid <= 0) return cudaSuccess;
    const CUtensorMap none{};
    const TmaPassArgs a0{};
    const TmaBatchArgs b0{};
    return launch_pdl(xpass_warp_kernel<N, VSEP, BATCH>, dim3(grid), dim3(G::THREADS), G::SMEM, s,
                      BATCH ? none : *ms, BATCH ? none : *mv, BATCH ? none : *md, BATCH ? a0 : *a, BATCH ? *ba : b0);
}

template <bool VSEP, bool BATCH>
cudaError_t red_xw_n(int N, const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md,
                     const TmaPassArgs *a, const TmaBatchArgs *ba, cudaStream_t s)
{
    switch (N) {
    case 32: return red_xw<32, VSEP, BATCH>(ms, mv, md, a, ba, s);
    case 48: return red_xw<48, VSEP, BATCH>(ms, mv, md, a, ba, s);
    case 64: return red_xw<64, VSEP, BATCH>(ms, mv, md, a, ba, s);
    case 96: return red_xw<96, VSEP, BATCH>(ms, mv, md, a, ba, s);
    case 128: return red_xw<128, VSEP, BATCH>(ms, mv, md, a, ba, s);
    case 256: return red_xw<256, VSEP, BATCH>(ms, mv, md, a, ba, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int P, int K, bool BATCH>
cudaError_t red_s(const CUtensorMap *ms, const CUtensorMap *md, const TmaPassArgs *a, const TmaBatchArgs *ba,
                  cudaStream_t s)
{
    constexpr int EX = tmared_e(N);
    using G = SRed<N, EX, P, K, BATCH>;
    int grid = 0;
    cudaError_t e = persistent_grid<spass_tmared_kernel<N, EX, P, K, BATCH>>(G::THREADS, G::SMEM, &grid);
    if (e != cudaSuccess || !(BATCH ? (const void *)ba : (const void *)a)) return e;
    const int total = BATCH ? ba->members * ba->tiles : a->n_tiles;
    if (total < grid) grid = total;
    if (grid <= 0) return cudaSuccess;
    const CUtensorMap none{};
    const TmaPassArgs a0{};
    const TmaBatchArgs b0{};
    return launch_pdl(spass_tmared_kernel<N, EX, P, K, BATCH>, dim3(grid), dim3(P, G::TT, K), G::SMEM, s,
                      BATCH ? none : *ms, BATCH ? none : *md, BATCH ? a0 : *a, BATCH ? *ba : b0);
}

// Strided pass of N points with P column pairs and K planes per tile (from
// tmared_pairs, tmared_planes: K is tmared_max_planes(N, P) or 1).
template <int N, int P, bool BATCH>
cudaError_t red_s_k(int K, const CUtensorMap *ms, const CUtensorMap *md, const TmaPassArgs *a,
                    const TmaBatchArgs *ba, cudaStream_t s)
{
    constexpr int KM = tmared_max_planes(N, P);
    if (K == KM) return red_s<N, P, KM, BATCH>(ms, md, a, ba, s);
    if constexpr (KM > 1) {
        if (K == 1) return red_s<N, P, 1, BATCH>(ms, md, a, ba, s);
    }
    return cudaErrorInvalidValue;
}

template <int N, bool BATCH>
cudaError_t red_s_p(int P, int K, const CUtensorMap *ms, const CUtensorMap *md, const TmaPassArgs *a,
                    const TmaBatchArgs *ba, cudaStream_t s)
{
    constexpr int PM = tmared_unit(N) / N;  // largest P of this line length
    switch (P) {
    case 8: return red_s_k<N, 8, BATCH>(K, ms, md, a, ba, s);
    case 16:
        if constexpr (PM >= 16) return red_s_k<N, 16, BATCH>(K, ms, md, a, ba, s);
        break;
    case 32:
        if constexpr (PM >= 32) return red_s_k<N, 32, BATCH>(K, ms, md, a, ba, s);
        break;
    case 64:
        if constexpr (PM >= 64) return red_s_k<N, 64, BATCH>(K, ms, md, a, ba, s);
        break;
    default: break;
    }
    return cudaErrorInvalidValue;
}

template <bool BATCH, bool VSEP>
cudaError_t red_x_n(int N, const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md, const TmaPassArgs *a,
                    const TmaBatchArgs *ba, cudaStream_t s)
{
    switch (N) {
    case 32: return red_x<32, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 64: return red_x<64, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 128: return red_x<128, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 256: return red_x<256, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 512: return red_x<512, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 48: return red_x<48, BATCH, VSEP>(ms, mv, md, a, ba, s);
    case 96: return red_x<96, BATCH, VSEP>(ms, mv, md, a, ba, s);
    default: return cudaErrorInvalidValue;
    }
}

template <bool BATCH>
cudaError_t red_any(int axis, int N, int64_t nx, int K, const CUtensorMap *ms, const CUtensorMap *mv,
                    const CUtensorMap *md, const TmaPassArgs *a, const TmaBatchArgs *ba, cudaStream_t s)
{
    if (!tmared_eligible(N)) return cudaErrorInvalidValue;
    if (axis == 0) {
        if (nx != N) return cudaErrorInvalidValue;
        // a separable potential takes the table form (a single grid with
        // a->vyz set; a batch whose members all have tables, ba->vsep); the
        // set-up call (no args) prepares both forms
        const bool setup = BATCH ? !ba : !a;
        if (setup) {
            const cudaError_t e = red_x_n<BATCH, true>(N, ms, mv, md, a, ba, s);
            if (e != cudaSuccess) return e;
        } else if constexpr (BATCH) {
            if (ba->vsep) return red_x_n<true, true>(N, ms, mv, md, a, ba, s);
        } else if (a->vyz) {
            if (!a->vx) return cudaErrorInvalidValue;
            return red_x_n<false, true>(N, ms, mv, md, a, ba, s);
        }
        return red_x_n<BATCH, false>(N, ms, mv, md, a, ba, s);
    }
    const int P = tmared_pairs(N, nx);
    switch (N) {
    case 32: return red_s_p<32, BATCH>(P, K, ms, md, a, ba, s);
    case 64: return red_s_p<64, BATCH>(P, K, ms, md, a, ba, s);
    case 128: return red_s_p<128, BATCH>(P, K, ms, md, a, ba, s);
    case 256: return red_s_p<256, BATCH>(P, K, ms, md, a, ba, s);
    case 512: return red_s_p<512, BATCH>(P, K, ms, md, a, ba, s);
    case 48: return red_s_p<48, BATCH>(P, K, ms, md, a, ba, s);
    case 96: return red_s_p<96, BATCH>(P, K, ms, md, a, ba, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, bool BATCH>
cudaError_t fxy_n(const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md, const TmaPassArgs *a,
                  const TmaBatchArgs *ba, cudaStream_t s)
{
    using G = FXy<N, BATCH>;
    int grid = 0;
    cudaError_t e = persistent_grid<fxy_tmared_kernel<N, BATCH>>(G::THREADS, G::SMEM, &grid);
    if (e != cudaSuccess || !(BATCH ? (const void *)ba : (const void *)a)) return e;
    const int total = BATCH ? ba->members * ba->tiles : a->n_tiles;
    if (total < grid) grid = total;
    if (grid <= 0) return cudaSuccess;
    const CUtensorMap none{};
    const TmaPassArgs a0{};
    const TmaBatchArgs b0{};
    return launch_pdl(fxy_tmared_kernel<N, BATCH>, dim3(grid), dim3(G::THREADS), G::SMEM, s,
                      BATCH ? none : *ms, BATCH ? none : *mv, BATCH ? none : *md, BATCH ? a0 : *a, BATCH ? *ba : b0);
}

template <bool BATCH>
cudaError_t fxy_any(int N, const CUtensorMap *ms, const CUtensorMap *mv, const CUtensorMap *md, const TmaPassArgs *a,
                    const TmaBatchArgs *ba, cudaStream_t s)
{
    switch (N) {
    case 32: return fxy_n<32, BATCH>(ms, mv, md, a, ba, s);
    case 64: return fxy_n<64, BATCH>(ms, mv, md, a, ba, s);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void separable_v_kernel(const float *vx, const float *vyz, float *V, int64_t nx, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        V[p] = __fadd_rn(vx[p % nx], vyz[p / nx]);
}

}  // namespace

cudaError_t build_separable_v(const float *vx, const float *vyz, float *V, int64_t nx, int64_t rows,
                              cudaStream_t s)
{
    const int64_t n = nx * rows;
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    separable_v_kernel<<<(unsigned)blocks, 256, 0, s>>>(vx, vyz, V, nx, n);
    return cudaGetLastError();
}

cudaError_t launch_pass_fxy(int N, const CUtensorMap &msrc, const CUtensorMap &mV, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s)
{
    return fxy_any<false>(N, &msrc, &mV, &mdst, &a, nullptr, s);
}

cudaError_t launch_pass_fxy_batch(int N, const TmaBatchArgs &a, cudaStream_t s)
{
    return fxy_any<true>(N, nullptr, nullptr, nullptr, nullptr, &a, s);
}

cudaError_t prepare_pass_fxy(int N, bool batch)
{
    return batch ? fxy_any<true>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr)
                 : fxy_any<false>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_pass_xwarp(int N, const CUtensorMap &msrc, const CUtensorMap &mV, const CUtensorMap &mdst,
                              const TmaPassArgs &a, cudaStream_t s)
{
    if (a.vyz) {
        if (!a.vx) return cudaErrorInvalidValue;
        return red_xw_n<true, false>(N, &msrc, &mV, &mdst, &a, nullptr, s);
    }
    return red_xw_n<false, false>(N, &msrc, &mV, &mdst, &a, nullptr, s);
}

cudaError_t prepare_pass_xwarp(int N)
{
    const cudaError_t e = red_xw_n<true, false>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return e != cudaSuccess ? e : red_xw_n<false, false>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_pass_xwarp_batch(int N, const TmaBatchArgs &a, cudaStream_t s)
{
    return a.vsep ? red_xw_n<true, true>(N, nullptr, nullptr, nullptr, nullptr, &a, s)
                  : red_xw_n<false, true>(N, nullptr, nullptr, nullptr, nullptr, &a, s);
}

cudaError_t prepare_pass_xwarp_batch(int N)
{
    const cudaError_t e = red_xw_n<true, true>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return e != cudaSuccess ? e : red_xw_n<false, true>(N, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_pass_tmared(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mV,
                               const CUtensorMap &mdst, const TmaPassArgs &a, cudaStream_t s)
{
    return red_any<false>(axis, N, a.nx, a.planes, &msrc, &mV, &mdst, &a, nullptr, s);
}

cudaError_t prepare_pass_tmared(int axis, int N, int64_t nx, int planes)
{
    return red_any<false>(axis, N, nx, planes, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_pass_tmared_batch(int axis, int N, const TmaBatchArgs &a, cudaStream_t s)
{
    return red_any<true>(axis, N, a.nx, a.planes, nullptr, nullptr, nullptr, nullptr, &a, s);
}

cudaError_t prepare_pass_tmared_batch(int axis, int N, int64_t nx, int planes)
{
    return red_any<true>(axis, N, nx, planes, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

}  // namespace spstd
