// pass_xy.cuh -- the x and y passes of a 3D FP32 half-stage in one persistent
// kernel, ordered plane by plane so that the second touch of every plane hits
// the L2 cache.
//
// Per half-stage the separate passes move src + V + 2 dst (x) and src + 2 dst
// (y) through HBM.  Here a plane's y tiles (dst += a L_y src) run first and
// its x tiles (dst += a L_x src + bV V src) a few planes later: the x tiles
// find that plane's src and freshly written dst still in L2, so HBM sees one
// read of src, V and dst and one write of dst for both passes.
//
// Schedule.  One work list, claimed item by item from a global counter (a
// block only ever holds items it is running): the y tiles of planes 0..D-1,
// then for each plane j its x tiles followed by the y tiles of plane j + D.
// With D (tiles per plane) well above the number of items the grid holds at
// once, an x tile's plane is normally finished when it is claimed.  Otherwise
// the x tile waits (bounded spin) until every y tile of its plane has been
// stored, counted on a per-plane counter with release/acquire.  A block never
// waits while it holds an unfinished y tile: an x claim made behind a y tile
// that is still in flight is deferred to the top of its own iteration, and the
// block claims nothing more until then; finished y tiles are counted before
// any wait.  Every claimed y tile is therefore held by a block that will
// finish it, and an x tile depends only on y tiles claimed before it, so every
// wait ends -- whatever part of the grid is resident.  The counters reset
// themselves (the last x tile of a plane, the last block to exit), so graph
// replays start clean.
#pragma once

#include "fft_line.cuh"
#include "pass_tma.cuh"

namespace spstd {

// An x tile waits for its plane at most this many polls, 64 ns of backoff
// each: about a second, far beyond any legitimate wait (a few microseconds).
constexpr uint32_t kMaxDepSpins = 1u << 20;

struct XyPassArgs {
    const float2 *twx, *twy;   // W_N tables of the x and y axes
    const float *multx, *multy;
    const float *V;
    float bV;
    int nx, ny, nz;
    int nyt;                   // y tiles per plane (nx / 32)
    int nxt;                   // x tiles per plane (ny / 32)
    int lag;                   // D: planes between a plane's y tiles and its x tiles in the list
    unsigned *claim;           // [0] items claimed, [1] blocks finished
    unsigned *ydone;           // [nz] y tiles stored per plane
    unsigned *xseen;           // [nz] x tiles of the plane past their wait
    int *status;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Publishes completed TMA stores: async-proxy writes before the release add.
__device__ __forceinline__ void release_add(unsigned *p)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

struct XyItem {
    int type;  // 0 y tile, 1 x tile, -1 past the end
    int plane;
    int tile;
};

// Item w of the work list.
__device__ __forceinline__ XyItem xy_item(const XyPassArgs &a, unsigned w)
{
    const int D = a.lag < a.nz ? a.lag : a.nz;
    const unsigned head = (unsigned)D * a.nyt;
    const unsigned S = (unsigned)(a.nxt + a.nyt);
    const unsigned body = (unsigned)(a.nz - D) * S;
    const unsigned total = head + body + (unsigned)D * a.nxt;
    if (w >= total) return {-1, 0, 0};
    if (w < head) return {0, (int)(w / a.nyt), (int)(w % a.nyt)};
    w -= head;
    if (w < body) {
        const int j = (int)(w / S), r = (int)(w % S);
        return r < a.nxt ? XyItem{1, j, r} : XyItem{0, j + D, r - a.nxt};
    }
    w -= body;
    return {1, a.nz - D + (int)(w / a.nxt), (int)(w % a.nxt)};
}

template <int N>
__host__ __device__ constexpr size_t xy_pass_smem()
{
    return (size_t)kTmaStages * 2 * kTmaRows * N * sizeof(float) + 2 * N * sizeof(float2) + 2 * N * sizeof(float) +
           kTmaStages * sizeof(int4) + 2 * kTmaStages * sizeof(uint64_t) + 1024;
}

// Barrier among the compute warps only (named barrier 1; the producer warp
// never joins it).
template <int NT>
__device__ __forceinline__ void compute_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Column exchange of a y tile ([N rows][16 pairs], pair p at column p) ordered
// by the compute-warp barrier.
template <int NT>
struct XcColNB {
    float2 *base;  // tile + p
    __device__ __forceinline__ float2 &at(int idx) { return base[idx * 16]; }
    __device__ __forceinline__ void st(int idx, float2 v) { at(idx) = v; }
    __device__ __forceinline__ float2 ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { compute_sync<NT>(); }
    __device__ __forceinline__ void flip() { compute_sync<NT>(); }
};

// N = nx = ny in {64, 128, 256}.  Block: 16 N/E compute threads (a tile as 16
// line pairs or 16 column pairs) and one producer warp.
//
// Warp specialisation.  Lane 0 of the producer warp claims the items, waits
// for x tiles' planes, starts the TMA loads of a stage (completion on
// full[s]), and, once the compute warps have finished a stage (done[s]),
// stores its dst tile and counts finished y tiles.  The compute warps only
// wait for full[s] and never for the producer's bookkeeping.  Before the
// producer waits on another block's y tiles it first stores and counts every
// item it holds (so no block waits while holding an unfinished y tile).
template <int N, int E>
__global__ void __launch_bounds__(16 * (N / E) + 32, 1)
xypass_tma_kernel(const __grid_constant__ CUtensorMap msx, const __grid_constant__ CUtensorMap mdx,
                  const __grid_constant__ CUtensorMap msy, const __grid_constant__ CUtensorMap mdy,
                  const XyPassArgs a)
{
    constexpr int TT = N / E;
    constexpr int NT = 16 * TT;  // compute threads
    constexpr uint32_t kTileBytes = kTmaRows * N * sizeof(float);
    static_assert(kTmaRows == kTmaCols, "x and y tiles share the stage buffers");
    static_assert(NT % 32 == 0, "whole compute warps");
    if (blockDim.x != NT + 32) {  // launched without its producer warp: refuse, do not wait
        if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
        return;
    }
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *s_src = reinterpret_cast<float *>(base);
    float *s_dst = s_src + kTmaStages * kTmaRows * N;
    float2 *twx = reinterpret_cast<float2 *>(s_dst + kTmaStages * kTmaRows * N);
    float2 *twy = twx + N;
    float *multx = reinterpret_cast<float *>(twy + N);
    float *multy = multx + N;
    int4 *ring = reinterpret_cast<int4 *>(multy + N);  // per stage: type (0 y, 1 x), plane, tile, valid
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + kTmaStages);
    uint64_t *done = full + kTmaStages;
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], 1);
        }
        mbar_fence_init();
        s_abort = 0;
    }
    for (int i = tid; i < N; i += NT + 32) {
        twx[i] = a.twx[i];
        twy[i] = a.twy[i];
        multx[i] = a.multx[i];
        multy[i] = a.multy[i];
    }
    __syncthreads();  // the last block-wide barrier: the roles split here

    if (tid >= NT) {
        // ================= producer warp (lane 0) =================
        if (tid != NT) return;
        int4 held[kTmaStages] = {};  // item of each stage, loaded and not yet stored
        int pend[kTmaStages + 1];   // planes of y tiles stored but not yet counted (oldest first)
        int npend = 0;
        bool newest_y = false;      // the newest committed store is the tail of pend
        bool ok = true;
        // Stores item j (stage j % 3) once the compute warps are done with it.
        auto store = [&](int j) {
            const int s = j % kTmaStages;
            if (!mbar_wait(&done[s], (uint32_t)((j / kTmaStages) & 1))) {
                atomicExch(a.status, kStatusTimeout);
                ok = false;
                return;
            }
            const int4 it = held[s];
            float *dst = s_dst + s * kTmaRows * N;
            if (it.x == 1)
                tma_store_3d(&mdx, 0, it.y * a.ny + it.z * kTmaRows, 0, dst);
            else
                tma_store_3d(&mdy, it.z * kTmaCols, 0, it.y, dst);
            bulk_commit();
            newest_y = it.x == 0;
            if (newest_y) pend[npend++] = it.y;
        };
        // Counts the y tiles whose stores are complete (all = wait for every store).
        auto count = [&](bool all) {
            if (npend == 0) return;
            if (all) {
                bulk_wait_all();
                for (int i = 0; i < npend; ++i) release_add(a.ydone + pend[i]);
                npend = 0;
                return;
            }
            // every store but the newest is complete; keep the newest if it is a pending y tile
            asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
            const int n = newest_y ? npend - 1 : npend;
            for (int i = 0; i < n; ++i) release_add(a.ydone + pend[i]);
            if (n > 0 && n < npend) pend[0] = pend[n];
            npend -= n;
        };
        int k = 0, kstore = 0;
        for (;; ++k) {
            const int s = k % kTmaStages;
            if (k >= kTmaStages) {
                // stage s held item k - 3: store it (unless a drain did), and let the
                // store read the tile before the stage is reloaded
                if (kstore <= k - kTmaStages) {
                    store(k - kTmaStages);
                    kstore = k - kTmaStages + 1;
                    if (!ok) break;
                }
                bulk_wait_read<0>();
                count(false);
            }
            const XyItem it = xy_item(a, atomicAdd(a.claim, 1u));
            if (it.type < 0) break;
            if (it.type == 1 && ld_acquire_gpu(a.ydone + it.plane) < (unsigned)a.nyt) {
                // hold nothing unfinished while waiting on other blocks' y tiles
                for (; kstore < k && ok; ++kstore) store(kstore);
                if (!ok) break;
                count(true);
                uint32_t spins = 0;
                while (ld_acquire_gpu(a.ydone + it.plane) < (unsigned)a.nyt) {
                    if (++spins > kMaxDepSpins) {
                        atomicExch(a.status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                    __nanosleep(64);
                }
                if (!ok) break;
            }
            if (it.type == 1) {
                fence_proxy_async_global();
                if (atomicAdd(a.xseen + it.plane, 1u) == (unsigned)a.nxt - 1) {
                    // every x tile of the plane is past its wait: reset for the next launch
                    a.ydone[it.plane] = 0;
                    a.xseen[it.plane] = 0;
                }
            }
            held[s] = make_int4(it.type, it.plane, it.tile, 1);
            ring[s] = held[s];
            mbar_arrive_expect_tx(&full[s], 2 * kTileBytes);
            if (it.type == 1) {
                const int row0 = it.plane * a.ny + it.tile * kTmaRows;
                tma_load_3d(s_src + s * kTmaRows * N, &msx, 0, row0, 0, &full[s]);
                tma_load_3d(s_dst + s * kTmaRows * N, &mdx, 0, row0, 0, &full[s]);
            } else {
                tma_load_3d(s_src + s * kTmaRows * N, &msy, it.tile * kTmaCols, 0, it.plane, &full[s]);
                tma_load_3d(s_dst + s * kTmaRows * N, &mdy, it.tile * kTmaCols, 0, it.plane, &full[s]);
            }
        }
        // end of the list (or a failure): mark stage k % 3 empty for the compute
        // warps (its previous item, k - 3, is stored: they are done with it), then
        // store what they are still finishing
        const int s_end = k % kTmaStages;
        ring[s_end] = make_int4(0, 0, 0, 0);
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s_end])) : "memory");
        for (; kstore < k && ok; ++kstore) store(kstore);
        count(true);
        bulk_wait_all();
        // the last block out resets the claim counters for the next launch
        if (atomicAdd(a.claim + 1, 1u) == gridDim.x - 1) {
            a.claim[0] = 0;
            a.claim[1] = 0;
        }
        return;
    }

    // ================= compute warps =================
    for (int k = 0;; ++k) {
        const int s = k % kTmaStages;
        const bool ok = mbar_wait(&full[s], (uint32_t)((k / kTmaStages) & 1));
        if (!ok) s_abort = 1;
        compute_sync<NT>();
        if (s_abort) {
            if (tid == 0) atomicExch(a.status, kStatusTimeout);
            break;
        }
        const int4 it = ring[s];
        if (!it.w) break;  // end of this block's items
        const int plane = it.y, tile = it.z;
        float *src = s_src + s * kTmaRows * N;
        float *dst = s_dst + s * kTmaRows * N;
        if (it.x == 1) {
            // x tile: 32 rows of the plane; the compute threads as (TT, 16) line pairs
            const int t = tid % TT, l = tid / TT;
            const int row0 = plane * a.ny + tile * kTmaRows;
            const int r0 = 2 * l, r1 = r0 + 1;
            float2 v[E], sv[E], Vv[E];
            const float *V0 = a.V + (int64_t)(row0 + r0) * N;
            const float *V1 = a.V + (int64_t)(row0 + r1) * N;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = t + e * TT;
                v[e] = make_float2(src[r0 * N + i], src[r1 * N + i]);
                sv[e] = v[e];
                Vv[e] = make_float2(__ldg(V0 + i), __ldg(V1 + i));
            }
            compute_sync<NT>();
            XcLine<N> xc{reinterpret_cast<float2 *>(src) + l * N};
            fft_line<float, N, E, false>(v, t, xc, twx);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float mm = multx[t + e * TT];
                v[e].x *= mm;
                v[e].y *= mm;
            }
            fft_line<float, N, E, true>(v, t, xc, twx);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = t + e * TT;
                dst[r0 * N + i] += fmaf(a.bV * Vv[e].x, sv[e].x, v[e].x);
                dst[r1 * N + i] += fmaf(a.bV * Vv[e].y, sv[e].y, v[e].y);
            }
        } else {
            // y tile: [N rows][16 column pairs]; the compute threads as (16, TT)
            const int p = tid % 16, t = tid / 16;
            float2 *src2 = reinterpret_cast<float2 *>(src);
            float2 *dst2 = reinterpret_cast<float2 *>(dst);
            float2 v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = src2[(t + e * TT) * 16 + p];
            compute_sync<NT>();
            XcColNB<NT> xc{src2 + p};
            fft_line<float, N, E, false>(v, t, xc, twy);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float mm = multy[t + e * TT];
                v[e].x *= mm;
                v[e].y *= mm;
            }
            fft_line<float, N, E, true>(v, t, xc, twy);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int q = (t + e * TT) * 16 + p;
                float2 d = dst2[q];
                d.x += v[e].x;
                d.y += v[e].y;
                dst2[q] = d;
            }
        }
        fence_proxy_async();
        compute_sync<NT>();
        if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&done[s])) : "memory");
    }
}

}  // namespace spstd
