// pass_tma.cuh -- stored-tile pipelined FP32 half-stage passes for line
// lengths 64..256 (schedule 5 and the fused x-y pass).
//
// One persistent block per SM walks its share of the tiles.  Thread 0 keeps
// the next tiles in flight with TMA bulk tensor loads into a 3-deep ring of
// shared-memory stages (src tile + dst tile per stage, completion on an
// mbarrier); the block transforms the current tile (same register/shared
// Stockham line FFT as the plain kernels, the consumed src tile doubling as
// the exchange buffer), adds the result into the dst tile in place and thread 0
// writes it back with a TMA bulk tensor store.  Loads run two tiles ahead, a
// store has one tile of slack before its stage is reloaded.
//
//   x pass:        tile = 32 contiguous rows of N points (16 complex line
//                  pairs), block (N/E, 16); also adds bV V src.
//   strided pass:  tile = N points along y or z x 32 adjacent x columns (16
//                  column pairs), block (16, N/E).
// E is the number of complex points a thread holds.
// Waits are bounded: on a timeout the block records kStatusTimeout, lets its
// stores drain and returns.
//
// These stored-tile kernels are schedule 5; the default kernels are the
// reduce-add passes of pass_tmared.cuh.
#pragma once

#include "fft_line.cuh"
#include "pass_tma_launch.h"
#include "tma.cuh"

namespace spstd {

constexpr int kTmaStages = 3;
constexpr int kTmaRows = 32;     // x pass: rows per tile
constexpr int kTmaCols = 32;     // strided pass: x columns per tile

// Line-private exchange region: line l owns N consecutive complex slots of
// the (already consumed) src tile, index XOR-swizzled within groups of 16 so
// that the scattered Stockham writes and the natural-layout reads of a
// 16-thread line hit 16 different 8-byte bank pairs.  The threads of a line
// sit in one warp, so a warp barrier orders the exchange; each read phase is
// closed by a second warp barrier (flip) before the next write phase.
// Column exchange inside a strided tile ([N rows][16 pairs], pair p at column
// p): a warp spans 16 consecutive pairs, so every access is a contiguous
// 128-byte row segment.  Block barriers order it; each read phase is closed by
// a second barrier (flip) before the next write phase, so the consumed src
// tile serves as the only buffer.
struct XcColB {
    float2 *base;  // tile + p
    __device__ __forceinline__ float2 &at(int idx) { return base[idx * 16]; }
    __device__ __forceinline__ void st(int idx, float2 v) { at(idx) = v; }
    __device__ __forceinline__ float2 ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    __device__ __forceinline__ void flip() { __syncthreads(); }
};

template <int N>
struct XcLine {
    float2 *base;  // region + line * N
    __device__ __forceinline__ float2 &at(int idx) { return base[idx ^ ((idx >> 4) & 15)]; }
    __device__ __forceinline__ void st(int idx, float2 v) { at(idx) = v; }
    __device__ __forceinline__ float2 ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { __syncwarp(); }
    __device__ __forceinline__ void flip() { __syncwarp(); }
};

// Bounded wait on a stage barrier by every thread, then a block vote: false if
// any thread timed out.  (Measured faster than one spinning thread plus a
// broadcast.)
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, int tid)
{
    const bool ok = mbar_wait(bar, parity);
    return !__syncthreads_or(!ok);
}

template <int N>
__host__ __device__ constexpr size_t tma_pass_smem()
{
    // NS x (src + dst) tiles of 32 x N floats, twiddles, multipliers, barriers
    return (size_t)kTmaStages * 2 * kTmaRows * N * sizeof(float) + N * sizeof(float2) + N * sizeof(float) +
           kTmaStages * sizeof(uint64_t) + 1024;
}

struct TmaSmem {
    float *src, *dst;
    float2 *tw;
    float *mult;
    uint64_t *full;
};

template <int N>
__device__ __forceinline__ TmaSmem tma_carve(unsigned char *raw)
{
    // 1024-byte alignment for the TMA destinations
    unsigned char *p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    TmaSmem m;
    m.src = reinterpret_cast<float *>(p);
    m.dst = m.src + kTmaStages * kTmaRows * N;
    m.tw = reinterpret_cast<float2 *>(m.dst + kTmaStages * kTmaRows * N);
    m.mult = reinterpret_cast<float *>(m.tw + N);
    m.full = reinterpret_cast<uint64_t *>(m.mult + N);
    return m;
}

template <int N>
__device__ __forceinline__ void tma_setup(const TmaSmem &m, const TmaPassArgs &a, int tid, int nthreads)
{
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&m.full[s], 1);
        mbar_fence_init();
    }
    for (int i = tid; i < N; i += nthreads) {
        m.tw[i] = a.tw[i];
        m.mult[i] = a.mult[i];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// x pass
// ---------------------------------------------------------------------------
template <int N, int E>
__global__ void __launch_bounds__(16 * (N / E), 1)
xpass_tma_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mdst,
                 const TmaPassArgs a)
{
    constexpr int TT = N / E;
    constexpr uint32_t kTileBytes = kTmaRows * N * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const TmaSmem m = tma_carve<N>(smem_raw);
    const int t = threadIdx.x, l = threadIdx.y, tid = l * TT + t;
    tma_setup<N>(m, a, tid, 16 * TT);

    const int nk = (int)blockIdx.x < a.n_tiles ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_of = [&](int k) {
        const int tile = (int)blockIdx.x + k * (int)gridDim.x;
        return a.reverse ? a.n_tiles - 1 - tile : tile;
    };
    auto issue = [&](int k) {
        const int s = k % kTmaStages;
        const int row0 = tile_of(k) * kTmaRows;
        mbar_arrive_expect_tx(&m.full[s], 2 * kTileBytes);
        tma_load_3d(m.src + s * kTmaRows * N, &msrc, 0, row0, 0, &m.full[s]);
        tma_load_3d(m.dst + s * kTmaRows * N, &mdst, 0, row0, 0, &m.full[s]);
    };
    if (tid == 0)
        for (int k = 0; k < kTmaStages - 1 && k < nk; ++k) issue(k);

    for (int k = 0; k < nk; ++k) {
        const int s = k % kTmaStages;
        if (!stage_wait(&m.full[s], (uint32_t)((k / kTmaStages) & 1), tid)) {
            if (tid == 0) {
                atomicExch(a.status, kStatusTimeout);
                bulk_wait_all();
            }
            return;
        }
        const int row0 = tile_of(k) * kTmaRows;
        float *src = m.src + s * kTmaRows * N;
        float *dst = m.dst + s * kTmaRows * N;
        const int r0 = 2 * l, r1 = 2 * l + 1;
        const bool ok0 = row0 + r0 < a.rows, ok1 = row0 + r1 < a.rows;
        float2 v[E], sv[E], Vv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = t + e * TT;
            v[e] = make_float2(src[r0 * N + i], src[r1 * N + i]);
            sv[e] = v[e];
        }
        if (a.use_V) {
            const float *V0 = a.V + (int64_t)(row0 + r0) * N;
            const float *V1 = a.V + (int64_t)(row0 + r1) * N;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = t + e * TT;
                Vv[e] = make_float2(ok0 ? __ldg(V0 + i) : 0.f, ok1 ? __ldg(V1 + i) : 0.f);
            }
        }
        __syncthreads();
        XcLine<N> xc{reinterpret_cast<float2 *>(src) + l * N};
        fft_line<float, N, E, false>(v, t, xc, m.tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float mm = m.mult[t + e * TT];
            v[e].x *= mm;
            v[e].y *= mm;
        }
        fft_line<float, N, E, true>(v, t, xc, m.tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = t + e * TT;
            float rx = v[e].x, ry = v[e].y;
            if (a.use_V) {
                rx = fmaf(a.bV * Vv[e].x, sv[e].x, rx);
                ry = fmaf(a.bV * Vv[e].y, sv[e].y, ry);
            }
            dst[r0 * N + i] += rx;
            dst[r1 * N + i] += ry;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&mdst, 0, row0, 0, dst);
            bulk_commit();
            if (k + kTmaStages - 1 < nk) {
                bulk_wait_read<1>();
                issue(k + kTmaStages - 1);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// strided pass (y or z)
// ---------------------------------------------------------------------------
template <int N, int E>
__global__ void __launch_bounds__(16 * (N / E), 1)
spass_tma_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mdst,
                 const TmaPassArgs a)
{
    constexpr int TT = N / E;
    constexpr uint32_t kTileBytes = kTmaCols * N * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const TmaSmem m = tma_carve<N>(smem_raw);
    // block (16, TT): a warp covers the 16 column pairs of two rows
    const int p = threadIdx.x, t = threadIdx.y, tid = t * 16 + p;
    tma_setup<N>(m, a, tid, 16 * TT);

    const int nk = (int)blockIdx.x < a.n_tiles ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto coords = [&](int k, int &x, int &y, int &z) {
        int tile = (int)blockIdx.x + k * (int)gridDim.x;
        if (a.reverse) tile = a.n_tiles - 1 - tile;
        const int outer = tile / a.n_xt;
        x = (tile - outer * a.n_xt) * kTmaCols;
        y = a.axis == 1 ? 0 : outer;
        z = a.axis == 1 ? outer : 0;
    };
    auto issue = [&](int k) {
        const int s = k % kTmaStages;
        int x, y, z;
        coords(k, x, y, z);
        mbar_arrive_expect_tx(&m.full[s], 2 * kTileBytes);
        tma_load_3d(m.src + s * kTmaCols * N, &msrc, x, y, z, &m.full[s]);
        tma_load_3d(m.dst + s * kTmaCols * N, &mdst, x, y, z, &m.full[s]);
    };
    if (tid == 0)
        for (int k = 0; k < kTmaStages - 1 && k < nk; ++k) issue(k);

    for (int k = 0; k < nk; ++k) {
        const int s = k % kTmaStages;
        if (!stage_wait(&m.full[s], (uint32_t)((k / kTmaStages) & 1), tid)) {
            if (tid == 0) {
                atomicExch(a.status, kStatusTimeout);
                bulk_wait_all();
            }
            return;
        }
        // tiles are [N rows][16 pairs] of float2
        float2 *src = reinterpret_cast<float2 *>(m.src + s * kTmaCols * N);
        float2 *dst = reinterpret_cast<float2 *>(m.dst + s * kTmaCols * N);
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = src[(t + e * TT) * 16 + p];
        __syncthreads();
        XcColB xc{src + p};
        fft_line<float, N, E, false>(v, t, xc, m.tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float mm = m.mult[t + e * TT];
            v[e].x *= mm;
            v[e].y *= mm;
        }
        fft_line<float, N, E, true>(v, t, xc, m.tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int q = (t + e * TT) * 16 + p;
            float2 d = dst[q];
            d.x += v[e].x;
            d.y += v[e].y;
            dst[q] = d;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            int x, y, z;
            coords(k, x, y, z);
            tma_store_3d(&mdst, x, y, z, dst);
            bulk_commit();
            if (k + kTmaStages - 1 < nk) {
                bulk_wait_read<1>();
                issue(k + kTmaStages - 1);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace spstd
