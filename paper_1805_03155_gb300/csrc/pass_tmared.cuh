// pass_tmared.cuh -- the default pipelined FP32 half-stage passes (lines of
// 32..512 points): TMA loads into shared-memory rings, a TMA reduce-add
// epilogue.
//
// The destination field never enters the SM.  A block computes its tile's
// contribution a L_d src (+ bV V src on the x pass, Eq. 16/18) into the
// consumed src tile, and a TMA reduce-add (cp.reduce.async.bulk.tensor .add)
// accumulates it into dst at L2.  Each dst element receives exactly one add
// per launch, so results are deterministic.  Without a dst tile a stage holds
// only src (and V on the x pass): two persistent blocks per SM, each with its
// own ring of up to 8 stages, keep loads in flight and overlap one block's
// barriers with the other's compute.
//
// Tile geometry (sizes are fixed per line length N so that every block has
// 128 (x) or 256 (strided) threads and a 16 KB / 32 KB tile part):
//   x pass:        ROWS = 4096/N contiguous rows of N points, ROWS/2 line
//                  pairs, block (N/E, ROWS/2), stage = src + V tiles; with a
//                  separable potential (single grids) stage = src tile + the
//                  tile's ROWS values of vyz, three blocks per SM;
//   strided pass:  K planes of N points along y or z x 2P adjacent x columns
//                  (P column pairs, P = min(4096/N, n_x/2); K = 256/(P N/E)
//                  planes, at least 1), block (P, N/E, K).
// Waits are bounded: on a timeout the block records kStatusTimeout, lets its
// bulk operations drain and returns.
//
// Batched forms run the tiles of many same-shaped members in one launch; each
// stage then also carries its member's multiplier row (bulk-copied on the
// stage barrier), because dt and the stage coefficient differ per member.
#pragma once

#include "fft_line.cuh"
#include "pass_tma_launch.h"
#include "tma.cuh"

namespace spstd {

constexpr size_t kTmaRedRing = 192 * 1024;  // shared memory for the rings of the blocks of one SM
constexpr int kRedBlocks = 2;               // persistent blocks per SM

// Ring stages: as many stages of PARTS tiles of TILE floats as fit
// kTmaRedRing / B (B blocks per SM), at most 8.
template <int TILE, int PARTS, int B>
__host__ __device__ constexpr int tmared_stages()
{
    return (int)(kTmaRedRing / B / ((size_t)PARTS * TILE * sizeof(float)) < 8
                     ? kTmaRedRing / B / ((size_t)PARTS * TILE * sizeof(float))
                     : 8);
}

// Shared memory of a block: S stages of PARTS tiles (plus, batched, a
// multiplier row per stage), then the twiddles (and, single-grid, the
// multipliers) and the barriers, with room for 1024-byte alignment.
template <int N, int TILE, int PARTS, int S, bool BATCH>
__host__ __device__ constexpr size_t tmared_smem()
{
    return (size_t)S * (PARTS * TILE + (BATCH ? N : 0)) * sizeof(float) + N * sizeof(float2) +
           (BATCH ? 0 : N * sizeof(float)) + S * sizeof(uint64_t) + 1024;
}

struct TmaRedSmem {
    float *src, *vt;  // [S] src tiles, [S] V tiles (x pass)
    float *mult;      // single-grid: one row; batched: [S] rows
    float2 *tw;
    uint64_t *full;
};

template <int N, int TILE, int PARTS, int S, bool BATCH>
__device__ __forceinline__ TmaRedSmem tmared_carve(unsigned char *raw)
{
    const uint32_t pad = (1024u - (smem_u32(raw) & 1023u)) & 1023u;
    TmaRedSmem m;
    m.src = reinterpret_cast<float *>(raw + pad);
    m.vt = m.src + S * TILE;
    m.mult = m.src + S * PARTS * TILE;
    m.tw = reinterpret_cast<float2 *>(m.mult + (BATCH ? S * N : N));
    m.full = reinterpret_cast<uint64_t *>(m.tw + N);
    return m;
}

// Block prologue: barriers, twiddles and (single grid) the multiplier row --
// tables that no kernel writes while steps run -- then the wait for the
// grids this launch depends on.  Launched with programmatic stream
// serialisation, the prologue overlaps the previous pass's last tiles; the
// wait returns once that grid has completed and its writes are visible (at
// once for an ordinary launch).  The launch then lets its own dependents be
// scheduled: they start as this grid's blocks exit and wait in turn.
template <int N, int S>
__device__ __forceinline__ void tmared_setup(const TmaRedSmem &m, const float2 *tw, const float *mult, int tid,
                                             int nthreads)
{
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&m.full[s], 1);
        mbar_fence_init();
    }
    for (int i = tid; i < N; i += nthreads) {
        m.tw[i] = tw[i];
        if (mult) m.mult[i] = mult[i];
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
}

// Column exchange inside a strided tile: element idx of a line sits rs
// complex slots after element idx - 1 (rs = P, or K P for a z tile of K
// planes); a warp spans consecutive pairs of one or more rows, so its accesses
// are contiguous row segments.  Block barriers order it; each read phase is
// closed by a second barrier (flip) before the next write phase.
struct XcColP {
    float2 *base;  // the line's first element
    int rs;
    __device__ __forceinline__ float2 &at(int idx) { return base[idx * rs]; }
    __device__ __forceinline__ void st(int idx, float2 v) { at(idx) = v; }
    __device__ __forceinline__ float2 ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    __device__ __forceinline__ void flip() { __syncthreads(); }
};

// Line-private exchange region of an x tile: line pair l owns N consecutive
// complex slots (its own two rows), index XOR-swizzled within groups of 16 so
// that a line's threads hit distinct 8-byte bank pairs; c (a multiple of the
// line's thread count) moves the line pairs that share a warp onto different
// bank pairs.  The threads of a line sit in one warp, so warp barriers order
// it.
template <int N>
struct XcLineR {
    float2 *base;  // tile + l * N complex slots
    int c;
    __device__ __forceinline__ float2 &at(int idx) { return base[idx ^ (((idx >> 4) & 15) ^ c)]; }
    __device__ __forceinline__ void st(int idx, float2 v) { at(idx) = v; }
    __device__ __forceinline__ float2 ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { __syncwarp(); }
    __device__ __forceinline__ void flip() { __syncwarp(); }
};

// v[e] <-> v[e ^ g] for a g below G (a power of two): conditional swaps bit by
// bit, as selects (g differs between the line pairs of one warp).
template <int E, int G>
__device__ __forceinline__ void xor_permute(float2 (&v)[E], int g)
{
#pragma unroll
    for (int m = 1; m < G; m <<= 1) {
        const bool f = (g & m) != 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (e & m) continue;
            const float2 a = v[e], b = v[e | m];
            v[e] = f ? b : a;
            v[e | m] = f ? a : b;
        }
    }
}

// Bounded wait on a stage barrier by every thread, then a block vote: false if
// any thread timed out.
__device__ __forceinline__ bool red_stage_wait(uint64_t *bar, uint32_t parity)
{
    const bool ok = mbar_wait(bar, parity);
    return !__syncthreads_or(!ok);
}

// Thread 0 after a timed-out wait on tile k of a ring of S stages, nk tiles:
// records the timeout, then waits (bounded) for the loads it issued for tiles
// k+1 .. k+S-2 and for its bulk reduces, so that nothing still writes into
// this block's shared memory when it returns.
template <int S>
__device__ __forceinline__ void red_timeout_exit(uint64_t *full, int k, int nk, int *status)
{
    atomicExch(status, kStatusTimeout);
    for (int j = k + 1; j <= k + S - 2 && j < nk; ++j) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1));
    bulk_wait_all();
}

// One x tile: line pair l (rows 2l, 2l+1 of the tile), thread t.  Reads src
// (and V), computes a L_x src (+ bV V src) with the multipliers mr[e] (of
// element t + e N/E) and leaves it in the src tile.  No block barrier inside:
// the rows of a line pair belong to its N/E threads (within one warp) alone.
//
// Rows are multiples of 32 floats apart (or, for 48-point lines, rows of two
// line pairs differ by a multiple of 32), so the G = 32/(N/E) line pairs of a
// warp would read and write the same banks.  Line pair g of its warp
// therefore moves element t + TT (e ^ g') through register slot e, g' = g mod
// GP with GP = min(G, the largest power of two dividing E), and the registers
// are permuted into the FFT's natural order (and back) in between.  (For E =
// 12, GP = 4: the XOR stays inside each aligned group of four slots; the 8
// line pairs of a 48-point warp then meet in pairs on a bank.)
// The V term stays in registers (w) from the loads to the final write.
// The two halves of an x tile, so that a fused kernel can run other work
// between them.  Load: this thread's elements of rows 2l, 2l+1 into v (in
// register-slot order) and the V term into w.  Finish: permute, FFT, k^2,
// inverse, permute back, and write v + w (+ yadd, another pass's contribution
// to the same elements, when given) into the src rows.
template <int N, int E>
struct XTile {
    static constexpr int TT = N / E;
    static_assert(TT <= 32, "a line's threads must share one warp (the exchange uses warp barriers)");
    static constexpr int G = TT >= 32 ? 1 : 32 / TT;
    static constexpr int GP = G < p2div(E) ? G : p2div(E);
    float2 v[E], w[E];
    int t, l, g;

    __device__ __forceinline__ int pos(int e) const { return t + ((TT * e) ^ (TT * g)); }

    __device__ __forceinline__ void load(const float *src, const float *vt, float bV, bool useV, int t_, int l_)
    {
        t = t_;
        l = l_;
        g = l & (GP - 1);
        const int r0 = 2 * l, r1 = 2 * l + 1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = pos(e);
            v[e] = make_float2(src[r0 * N + i], src[r1 * N + i]);
            // rounded products (no contraction into the final add), so that every
            // instantiation of this tile rounds alike
            w[e] = useV ? make_float2(__fmul_rn(__fmul_rn(bV, vt[r0 * N + i]), v[e].x),
                                      __fmul_rn(__fmul_rn(bV, vt[r1 * N + i]), v[e].y))
                        : make_float2(0.f, 0.f);
        }
    }

    // As load, for a separable potential: the V term of row r at x index i is
    // vx[i] + vyz_r rounded to FP32 -- the value the V field holds for such a
    // potential -- so both forms give the same bits.
    __device__ __forceinline__ void load_sep(const float *src, const float *vx, float vyz0, float vyz1, float bV,
                                             int t_, int l_)
    {
        t = t_;
        l = l_;
        g = l & (GP - 1);
        const int r0 = 2 * l, r1 = 2 * l + 1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = pos(e);
            v[e] = make_float2(src[r0 * N + i], src[r1 * N + i]);
            const float x = vx[i];
            w[e] = make_float2(__fmul_rn(__fmul_rn(bV, __fadd_rn(x, vyz0)), v[e].x),
                               __fmul_rn(__fmul_rn(bV, __fadd_rn(x, vyz1)), v[e].y));
        }
    }

    __device__ __forceinline__ void finish(float *src, const float (&mr)[E], const float2 *tw, const float *yadd)
    {
        const int r0 = 2 * l, r1 = 2 * l + 1;
        xor_permute<E, GP>(v, g);
        // exchange swizzle: line pairs of a warp on different bank pairs
        const int gx = l & (G - 1);
        XcLineR<N> xc{reinterpret_cast<float2 *>(src) + l * N, TT < 16 ? (gx & (16 / TT - 1)) * TT : 0};
        fft_line<float, N, E, false>(v, t, xc, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            v[e].x *= mr[e];
            v[e].y *= mr[e];
        }
        fft_line<float, N, E, true>(v, t, xc, tw);
        xor_permute<E, GP>(v, g);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = pos(e);
            float a = __fadd_rn(v[e].x, w[e].x), b = __fadd_rn(v[e].y, w[e].y);
            if (yadd) {
                a = __fadd_rn(a, yadd[r0 * N + i]);
                b = __fadd_rn(b, yadd[r1 * N + i]);
            }
            src[r0 * N + i] = a;
            src[r1 * N + i] = b;
        }
    }
};

template <int N, int E>
__device__ __forceinline__ void xred_tile(float *src, const float *vt, const float (&mr)[E], const float2 *tw,
                                          float bV, bool useV, int t, int l)
{
    XTile<N, E> x;
    x.load(src, vt, bV, useV, t, l);
    x.finish(src, mr, tw, nullptr);
}

// One line of a strided tile (its first element at `line`, consecutive
// elements rs complex slots apart), thread t.  Computes a L_d src and leaves
// it in the tile.  Contains block barriers (the column exchange spans the
// block).  The line's values may come from another buffer of the same layout
// (`in`); `line` then serves only as exchange space and result.
template <int N, int E>
__device__ __forceinline__ void sred_tile(const float2 *in, float2 *line, int rs, const float *mult, const float2 *tw,
                                          int t)
{
    constexpr int TT = N / E;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = in[(t + e * TT) * rs];
    __syncthreads();
    XcColP xc{line, rs};
    fft_line<float, N, E, false>(v, t, xc, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const float mm = mult[t + e * TT];
        v[e].x *= mm;
        v[e].y *= mm;
    }
    fft_line<float, N, E, true>(v, t, xc, tw);
    // the inverse's last exchange ended with a block barrier: the tile is free
#pragma unroll
    for (int e = 0; e < E; ++e) line[(t + e * TT) * rs] = v[e];
}

// Where tile g of a launch is: member i (0 for a single grid) and the 4D
// coordinates of its box.  The maps split the line axis into (L1, L2) =
// (min(N, 256), N / L1) so that no box dimension exceeds 256:
//   x view  (x_lo, x_hi, row, 1)      box (L1, L2, ROWS, 1)   smem [ROWS][N]
//   y view  (x, y_lo, y_hi, z)        box (2P, L1, L2, K)     smem [K][N][2P]
//   z view  (x, y, z_lo, z_hi)        box (2P, K, L1, L2)     smem [N][K][2P]
struct TileAt {
    int i, c[4];
};

__device__ __forceinline__ TileAt tile_at_x(int g, int tiles, int rows, int reverse, int total)
{
    if (reverse) g = total - 1 - g;
    TileAt a;
    a.i = g / tiles;
    a.c[0] = 0;
    a.c[1] = 0;
    a.c[2] = (g - a.i * tiles) * rows;
    a.c[3] = 0;
    return a;
}

// Strided tiles hold K consecutive planes of the outer axis (z for the y
// pass, y for the z pass).
__device__ __forceinline__ TileAt tile_at_s(int g, int tiles, int n_xt, int cols, int K, int axis, int reverse,
                                            int total)
{
    if (reverse) g = total - 1 - g;
    TileAt a;
    a.i = g / tiles;
    const int lt = g - a.i * tiles;
    const int outer = lt / n_xt;
    a.c[0] = (lt - outer * n_xt) * cols;
    a.c[1] = axis == 1 ? 0 : outer * K;
    a.c[2] = 0;
    a.c[3] = axis == 1 ? outer * K : 0;
    return a;
}

__device__ __forceinline__ void load_tile(void *smem, const CUtensorMap *map, const TileAt &c, uint64_t *bar)
{
    tma_load_4d(smem, map, c.c[0], c.c[1], c.c[2], c.c[3], bar);
}

// V tiles: read once per pass, so loaded with the evict-first L2 policy.
__device__ __forceinline__ void load_v_tile(void *smem, const CUtensorMap *map, const TileAt &c, uint64_t *bar)
{
    tma_load_4d_hint(smem, map, c.c[0], c.c[1], c.c[2], c.c[3], bar, l2_evict_first_policy());
}

__device__ __forceinline__ void reduce_tile(const CUtensorMap *map, const TileAt &c, const void *smem)
{
    tma_reduce_add_4d(map, c.c[0], c.c[1], c.c[2], c.c[3], smem);
}

// ---------------------------------------------------------------------------
// x pass.  Single grid (BATCH = false): maps msrc / mV / mdst, a.mult, a.bV.
// Batched: member i's maps in ba.mem[i], its multipliers and bV in ba.pa[i].
// ---------------------------------------------------------------------------
template <int N, int E, bool BATCH, bool VSEP = false>
struct XRed {
    static constexpr int TT = N / E;
    static constexpr int ROWS = tmared_rows_x(N);
    static constexpr int LP = ROWS / 2;
    static constexpr int THREADS = LP * TT;
    static constexpr int TILE = ROWS * N;
    // stage: src (+ V) tile; with a separable potential, src and the tile's
    // ROWS values of vyz, so more stages fit (single grids: three blocks per
    // SM; batched, a stage also carries its member's multiplier and vx rows,
    // and the stages are counted with them)
    static constexpr int PARTS = VSEP ? 1 : 2;
    static constexpr int BLOCKS = VSEP ? 3 : kRedBlocks;
    static constexpr size_t SEP_STAGE = (size_t)(TILE + 2 * N + ROWS) * sizeof(float);
    static constexpr int S = !(BATCH && VSEP) ? tmared_stages<TILE, PARTS, BLOCKS>()
                             : kTmaRedRing / BLOCKS / SEP_STAGE < 8 ? (int)(kTmaRedRing / BLOCKS / SEP_STAGE) : 8;
    // vyz values [S][ROWS], then vx (one row; batched [S] rows)
    static constexpr size_t SEP_SMEM =
        VSEP ? 16 + (size_t)S * ROWS * sizeof(float) + (BATCH ? S : 1) * (size_t)N * sizeof(float) : 0;
    static constexpr size_t SMEM = tmared_smem<N, TILE, PARTS, S, BATCH>() + SEP_SMEM;
};

template <int N, int E, bool BATCH, bool VSEP = false>
__global__ void __launch_bounds__(XRed<N, E, BATCH, VSEP>::THREADS, XRed<N, E, BATCH, VSEP>::BLOCKS)
xpass_tmared_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mV,
                    const __grid_constant__ CUtensorMap mdst, const TmaPassArgs a, const TmaBatchArgs ba)
{
    using G = XRed<N, E, BATCH, VSEP>;
    constexpr int TT = G::TT, ROWS = G::ROWS, TILE = G::TILE, S = G::S;
    constexpr uint32_t kTileBytes = TILE * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const TmaRedSmem m = tmared_carve<N, TILE, G::PARTS, S, BATCH>(smem_raw);
    const int t = threadIdx.x, l = threadIdx.y, tid = l * TT + t;
    // separable potential: [S][ROWS] vyz values (one bulk copy per stage), then
    // vx (single grid: one row; batched: [S] rows, the tile's member's)
    float *vrow = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(m.full + S) + 15) & ~uintptr_t(15));
    float *vxt = vrow + S * ROWS;
    if constexpr (VSEP && !BATCH)
        for (int i = tid; i < N; i += G::THREADS) vxt[i] = a.vx[i];
    tmared_setup<N, S>(m, BATCH ? ba.tw : a.tw, BATCH ? nullptr : a.mult, tid, G::THREADS);
    const bool useV = BATCH || VSEP || a.use_V != 0;
    const int fsrc = BATCH ? (ba.src >= 0 ? ba.src : 1 - ba.dst) : 0;
    // single grid: one multiplier row for every tile, held in registers
    float mrow[E];
#pragma unroll
    for (int e = 0; e < E; ++e) mrow[e] = BATCH ? 0.f : m.mult[t + e * TT];

    const int tiles = BATCH ? ba.tiles : a.n_tiles;
    const int total = BATCH ? ba.members * ba.tiles : a.n_tiles;
    const int reverse = BATCH ? 0 : a.reverse;
    const int nk = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto at = [&](int k) { return tile_at_x((int)blockIdx.x + k * (int)gridDim.x, tiles, ROWS, reverse, total); };
    auto issue = [&](int k) {
        const int s = k % S;
        const TileAt c = at(k);
        if constexpr (BATCH) {
            const TmaMember *mm = ba.mem + c.i;
            const PassArgs<float> &pm = ba.pa[c.i];
            if constexpr (VSEP) {
                mbar_arrive_expect_tx(&m.full[s], kTileBytes + (2 * N + ROWS) * sizeof(float));
                load_tile(m.src + s * TILE, &mm->x[fsrc], c, &m.full[s]);
                bulk_load(vrow + s * ROWS, pm.vyz + c.c[2], ROWS * sizeof(float), &m.full[s]);
                bulk_load(vxt + s * N, pm.vx, N * sizeof(float), &m.full[s]);
            } else {
                mbar_arrive_expect_tx(&m.full[s], 2 * kTileBytes + N * sizeof(float));
                load_tile(m.src + s * TILE, &mm->x[fsrc], c, &m.full[s]);
                load_v_tile(m.vt + s * TILE, &mm->x[3], c, &m.full[s]);
            }
            bulk_load(m.mult + s * N, pm.mult, N * sizeof(float), &m.full[s]);
        } else {
            mbar_arrive_expect_tx(&m.full[s], VSEP ? kTileBytes + ROWS * sizeof(float) : (useV ? 2 : 1) * kTileBytes);
            // failure-path test hook: the launch's first tile may be left unloaded
            // (its barrier then never completes and the wait on it times out)
            if (k == 0 && blockIdx.x == 0 && a.inject && atomicExch(a.inject, 0) != 0) return;
            load_tile(m.src + s * TILE, &msrc, c, &m.full[s]);
            if constexpr (VSEP)
                bulk_load(vrow + s * ROWS, a.vyz + c.c[2], ROWS * sizeof(float), &m.full[s]);
            else if (useV)
                load_v_tile(m.vt + s * TILE, &mV, c, &m.full[s]);
        }
    };
    if (tid == 0)
        for (int k = 0; k < S - 1 && k < nk; ++k) issue(k);

    for (int k = 0; k < nk; ++k) {
        const int s = k % S;
        const TileAt c = at(k);
        if (!red_stage_wait(&m.full[s], (uint32_t)((k / S) & 1))) {
            if (tid == 0) red_timeout_exit<S>(m.full, k, nk, BATCH ? ba.mem[c.i].status : a.status);
            return;
        }
        float *src = m.src + s * TILE;
        if constexpr (BATCH) {
            // this tile's member's multipliers, from the row its stage carries
            float mr[E];
#pragma unroll
            for (int e = 0; e < E; ++e) mr[e] = m.mult[s * N + t + e * TT];
            if constexpr (VSEP) {
                XTile<N, E> x;
                x.load_sep(src, vxt + s * N, vrow[s * ROWS + 2 * l], vrow[s * ROWS + 2 * l + 1], ba.pa[c.i].bV, t, l);
                x.finish(src, mr, m.tw, nullptr);
            } else {
                xred_tile<N, E>(src, m.vt + s * TILE, mr, m.tw, ba.pa[c.i].bV, true, t, l);
            }
        } else if constexpr (VSEP) {
            XTile<N, E> x;
            x.load_sep(src, vxt, vrow[s * ROWS + 2 * l], vrow[s * ROWS + 2 * l + 1], a.bV, t, l);
            x.finish(src, mrow, m.tw, nullptr);
        } else {
            xred_tile<N, E>(src, m.vt + s * TILE, mrow, m.tw, a.bV, useV, t, l);
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            reduce_tile(BATCH ? &ba.mem[c.i].x[ba.dst] : &mdst, c, src);
            bulk_commit();
            if (k + S - 1 < nk) {
                bulk_wait_read<1>();
                issue(k + S - 1);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// x pass with per-warp tiles (schedule 6; N in {32, 48, 64, 96, 128, 256};
// single grids and batches).  The block pass above waits at two block
// barriers per tile (the stage vote and the hand-over to the thread that
// issues the reduce-add), so a warp that finishes its line pairs early idles
// until the slowest warp of the block is done.  Here each warp owns a ring of
// S stages of its own tiles -- the 2 (32/TT) rows of its line pairs, 3-4 KB of
// src (plus V, or the rows' vyz values for a separable potential; batched,
// also the tile's member's multiplier row and, with tables, its vx row) --
// with its own mbarriers; lane 0 issues the warp's loads and reduce-adds, and
// the lanes meet only at warp barriers.  The arithmetic of a tile (XTile) is
// the block pass's, so both give the same bits.  Waits are bounded per warp;
// a warp whose wait runs out records the timeout, drains its own loads and
// reduce-adds and returns.
// ---------------------------------------------------------------------------
template <int N, bool VSEP, bool BATCH = false>
struct XWarp {
    static constexpr int E = line_e<float, N>::value, TT = N / E;
    static_assert(TT >= 2 && TT <= 16, "per-warp x tiles take lines of 2..16 threads");
    static constexpr int LPW = 32 / TT;          // line pairs per warp
    static constexpr int ROWS = 2 * LPW;         // rows per warp tile
    static constexpr int TILE = ROWS * N;        // floats: 1024 (4 KB), 768 for 3 * 2^k lines
    static constexpr int WARPS = 4;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PARTS = VSEP ? 1 : 2;   // src (and V) per stage
    static constexpr int BLOCKS = VSEP ? 3 : 2;
    // floats of a warp's stage: its tiles, the rows' vyz values (tables) and,
    // batched, the member's multiplier row and vx row (tables)
    static constexpr int STAGE = PARTS * TILE + (VSEP ? ROWS : 0) + (BATCH ? (VSEP ? 2 : 1) * N : 0);
    // single grids count the tiles alone (the vyz values fit beside them)
    static constexpr size_t RING_UNIT = (size_t)(BATCH ? STAGE : PARTS * TILE) * sizeof(float);
    static constexpr int S0 = (int)(kTmaRedRing / BLOCKS / WARPS / RING_UNIT);
    static constexpr int S = S0 < 8 ? S0 : 8;
    static_assert(S >= 2, "a warp's ring needs two stages");
    static constexpr size_t SMEM = (size_t)WARPS * S * STAGE * sizeof(float) + (VSEP && !BATCH ? N * sizeof(float) : 0) +
                                   N * sizeof(float2) + N * sizeof(float) + (size_t)WARPS * S * sizeof(uint64_t) + 1024;
};

template <int N, bool VSEP, bool BATCH>
__global__ void __launch_bounds__(XWarp<N, VSEP, BATCH>::THREADS, XWarp<N, VSEP, BATCH>::BLOCKS)
xpass_warp_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mV,
                  const __grid_constant__ CUtensorMap mdst, const TmaPassArgs a, const TmaBatchArgs ba)
{
    using G = XWarp<N, VSEP, BATCH>;
    constexpr int E = G::E, TT = G::TT, ROWS = G::ROWS, TILE = G::TILE, S = G::S, W = G::WARPS;
    constexpr uint32_t kTileBytes = TILE * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    float *tbuf = reinterpret_cast<float *>(smem_raw + pad);   // [W][S][PARTS][TILE]
    float *vrows = tbuf + (size_t)W * S * G::PARTS * TILE;     // tables: [W][S][ROWS]
    float *brows = vrows + (VSEP ? W * S * ROWS : 0);          // batched: [W][S][N] multipliers, then vx
    float *vxt = brows + (BATCH ? (VSEP ? 2 : 1) * W * S * N : 0);  // single grid with tables: vx[N]
    float2 *tw = reinterpret_cast<float2 *>(vxt + (VSEP && !BATCH ? N : 0));
    float *mult = reinterpret_cast<float *>(tw + N);           // single grid: the multiplier row
    uint64_t *full_all = reinterpret_cast<uint64_t *>(mult + N);  // [W][S]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int t = lane % TT, l = lane / TT;
    uint64_t *full = full_all + w * S;
    float *wt = tbuf + (size_t)w * S * G::PARTS * TILE;
    float *wv = vrows + w * S * ROWS;
    float *wm = brows + w * S * N;            // batched: this warp's multiplier rows
    float *wx = brows + (W + w) * S * N;      // batched, tables: this warp's vx rows
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    for (int i = tid; i < N; i += G::THREADS) {
        if constexpr (BATCH) {
            tw[i] = ba.tw[i];
        } else {
            tw[i] = a.tw[i];
            mult[i] = a.mult[i];
            if constexpr (VSEP) vxt[i] = a.vx[i];
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
    float mrow[E];
#pragma unroll
    for (int e = 0; e < E; ++e) mrow[e] = BATCH ? 0.f : mult[t + e * TT];
    const bool useV = BATCH || VSEP || a.use_V != 0;
    const int fsrc = BATCH ? (ba.src >= 0 ? ba.src : 1 - ba.dst) : 0;

    // tile g: member g / tiles (0 for a single grid), rows from (g mod tiles) ROWS
    const int tiles = BATCH ? ba.tiles : a.n_tiles;
    const int total = BATCH ? ba.members * ba.tiles : a.n_tiles;
    const int gw = (int)blockIdx.x * W + w, nw = (int)gridDim.x * W;
    const int nk = gw < total ? (total - 1 - gw) / nw + 1 : 0;
    auto at = [&](int k) {
        int g = gw + k * nw;
        if (!BATCH && a.reverse) g = total - 1 - g;
        TileAt c;
        c.i = BATCH ? g / tiles : 0;
        c.c[0] = 0;
        c.c[1] = 0;
        c.c[2] = (g - c.i * tiles) * ROWS;
        c.c[3] = 0;
        return c;
    };
    auto issue = [&](int k) {
        const int s = k % S;
        const TileAt c = at(k);
        float *st = wt + (size_t)s * G::PARTS * TILE;
        if constexpr (BATCH) {
            const TmaMember *mm = ba.mem + c.i;
            const PassArgs<float> &pm = ba.pa[c.i];
            mbar_arrive_expect_tx(&full[s], kTileBytes + (VSEP ? (ROWS + N) * sizeof(float) : kTileBytes) +
                                                N * sizeof(float));
            load_tile(st, &mm->xw[fsrc], c, &full[s]);
            if constexpr (VSEP) {
                bulk_load(wv + s * ROWS, pm.vyz + c.c[2], ROWS * sizeof(float), &full[s]);
                bulk_load(wx + s * N, pm.vx, N * sizeof(float), &full[s]);
            } else {
                load_v_tile(st + TILE, &mm->xw[3], c, &full[s]);
            }
            bulk_load(wm + s * N, pm.mult, N * sizeof(float), &full[s]);
        } else {
            mbar_arrive_expect_tx(&full[s], VSEP ? kTileBytes + ROWS * sizeof(float) : (useV ? 2 : 1) * kTileBytes);
            // failure-path test hook: the first tile of the grid's first warp may be left unloaded
            if (k == 0 && gw == 0 && a.inject && atomicExch(a.inject, 0) != 0) return;
            load_tile(st, &msrc, c, &full[s]);
            if constexpr (VSEP)
                bulk_load(wv + s * ROWS, a.vyz + c.c[2], ROWS * sizeof(float), &full[s]);
            else if (useV)
                load_v_tile(st + TILE, &mV, c, &full[s]);
        }
    };
    if (lane == 0)
        for (int k = 0; k < S - 1 && k < nk; ++k) issue(k);
    __syncwarp();

    for (int k = 0; k < nk; ++k) {
        const int s = k % S;
        const TileAt c = at(k);
        const bool ok = mbar_wait(&full[s], (uint32_t)((k / S) & 1));
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) red_timeout_exit<S>(full, k, nk, BATCH ? ba.mem[c.i].status : a.status);
            return;
        }
        float *src = wt + (size_t)s * G::PARTS * TILE;
        XTile<N, E> x;
        if constexpr (BATCH) {
            // the tile's member: its multipliers and bV
            float mr[E];
#pragma unroll
            for (int e = 0; e < E; ++e) mr[e] = wm[s * N + t + e * TT];
            const float bV = ba.pa[c.i].bV;
            if constexpr (VSEP)
                x.load_sep(src, wx + s * N, wv[s * ROWS + 2 * l], wv[s * ROWS + 2 * l + 1], bV, t, l);
            else
                x.load(src, src + TILE, bV, true, t, l);
            x.finish(src, mr, tw, nullptr);
        } else {
            if constexpr (VSEP)
                x.load_sep(src, vxt, wv[s * ROWS + 2 * l], wv[s * ROWS + 2 * l + 1], a.bV, t, l);
            else
                x.load(src, src + TILE, a.bV, useV, t, l);
            x.finish(src, mrow, tw, nullptr);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            reduce_tile(BATCH ? &ba.mem[c.i].xw[ba.dst] : &mdst, c, src);
            bulk_commit();
            if (k + S - 1 < nk) {
                bulk_wait_read<1>();
                issue(k + S - 1);
            }
        }
        __syncwarp();
    }
    if (lane == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// strided pass (y or z), P column pairs per tile.
// ---------------------------------------------------------------------------
template <int N, int E, int P, int K, bool BATCH>
struct SRed {
    static constexpr int TT = N / E;
    static constexpr int THREADS = P * TT * K;
    static constexpr int TILE = 2 * P * N * K;
    static constexpr int S = tmared_stages<TILE, 1, kRedBlocks>();
    static constexpr size_t SMEM = tmared_smem<N, TILE, 1, S, BATCH>();
};

// block (P, N/E, K): column pair p of plane k.
template <int N, int E, int P, int K, bool BATCH>
__global__ void __launch_bounds__(SRed<N, E, P, K, BATCH>::THREADS, kRedBlocks)
spass_tmared_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mdst,
                    const TmaPassArgs a, const TmaBatchArgs ba)
{
    using G = SRed<N, E, P, K, BATCH>;
    constexpr int TILE = G::TILE, S = G::S;
    constexpr uint32_t kTileBytes = TILE * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const TmaRedSmem m = tmared_carve<N, TILE, 1, S, BATCH>(smem_raw);
    const int p = threadIdx.x, t = threadIdx.y, k = threadIdx.z;
    const int tid = (k * G::TT + t) * P + p;
    tmared_setup<N, S>(m, BATCH ? ba.tw : a.tw, BATCH ? nullptr : a.mult, tid, G::THREADS);
    const int axis = BATCH ? ba.axis : a.axis;
    const int fsrc = BATCH ? (ba.src >= 0 ? ba.src : 1 - ba.dst) : 0;
    // this thread's line in a tile, and the distance between its elements
    const int line0 = K == 1 ? p : (axis == 1 ? k * N * P + p : k * P + p);
    const int rs = K == 1 ? P : (axis == 1 ? P : K * P);

    const int tiles = BATCH ? ba.tiles : a.n_tiles;
    const int n_xt = BATCH ? ba.n_xt : a.n_xt;
    const int total = BATCH ? ba.members * ba.tiles : a.n_tiles;
    const int reverse = BATCH ? 0 : a.reverse;
    const int nk = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto at = [&](int kk) {
        return tile_at_s((int)blockIdx.x + kk * (int)gridDim.x, tiles, n_xt, 2 * P, K, axis, reverse, total);
    };
    auto view = [&](int i, int f) -> const CUtensorMap * {
        return axis == 1 ? &ba.mem[i].y[f] : &ba.mem[i].z[f];
    };
    auto issue = [&](int kk) {
        const int s = kk % S;
        const TileAt c = at(kk);
        if constexpr (BATCH) {
            mbar_arrive_expect_tx(&m.full[s], kTileBytes + N * sizeof(float));
            load_tile(m.src + s * TILE, view(c.i, fsrc), c, &m.full[s]);
            bulk_load(m.mult + s * N, ba.pa[c.i].mult, N * sizeof(float), &m.full[s]);
        } else {
            mbar_arrive_expect_tx(&m.full[s], kTileBytes);
            load_tile(m.src + s * TILE, &msrc, c, &m.full[s]);
        }
    };
    if (tid == 0)
        for (int kk = 0; kk < S - 1 && kk < nk; ++kk) issue(kk);

    for (int kk = 0; kk < nk; ++kk) {
        const int s = kk % S;
        const TileAt c = at(kk);
        if (!red_stage_wait(&m.full[s], (uint32_t)((kk / S) & 1))) {
            if (tid == 0) red_timeout_exit<S>(m.full, kk, nk, BATCH ? ba.mem[c.i].status : a.status);
            return;
        }
        float2 *src = reinterpret_cast<float2 *>(m.src + s * TILE);
        sred_tile<N, E>(src + line0, src + line0, rs, BATCH ? m.mult + s * N : m.mult, m.tw, t);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            reduce_tile(BATCH ? view(c.i, ba.dst) : &mdst, c, src);
            bulk_commit();
            if (kk + S - 1 < nk) {
                bulk_wait_read<1>();
                issue(kk + S - 1);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Fused x + y pass for grids with nx = ny = N in {32, 64}.  A unit of
// K = 4096/N^2 planes (16 KB, layout [K][N (y)][N (x)]) holds whole x lines
// and whole y lines, so both transforms run on it in shared memory and one
// TMA reduce-add writes the sum of the x term, the V term and the y term:
// HBM carries src, V and dst once for the two passes (16 B per point instead
// of 28).  128 threads, two blocks per SM, the same 3-stage ring as the x
// pass.  Per unit:
//   1. the x threads load their row-pair elements and the V term (registers);
//   2. the y threads read their column lines from src and transform them
//      with the V tile (no longer needed) as exchange space and result;
//   3. the x transform runs in the src rows and adds the V term and the y
//      result to each element; the unit is reduce-added into dst.
// The rounding order (x + V, then + y) differs from the separate passes
// (x + V into dst, then y), so results agree to FP32 rounding.
// ---------------------------------------------------------------------------
template <int N, bool BATCH>
struct FXy {
    static constexpr int E = 16, TT = N / E, P = N / 2, K = fxy_planes(N);
    static constexpr int THREADS = P * TT * K;  // also (K N / 2) line pairs x TT
    static constexpr int UNIT = K * N * N;
    static constexpr int S = tmared_stages<UNIT, 2, kRedBlocks>();
    static constexpr size_t SMEM = (size_t)S * (2 * UNIT + (BATCH ? 2 * N : 0)) * sizeof(float) +
                                   N * sizeof(float2) + (BATCH ? 0 : 2 * N * sizeof(float)) +
                                   S * sizeof(uint64_t) + 1024;
    static_assert(THREADS == K * N / 2 * TT, "the x and y mappings use the same threads");
};

template <int N, bool BATCH>
__global__ void __launch_bounds__(FXy<N, BATCH>::THREADS, kRedBlocks)
fxy_tmared_kernel(const __grid_constant__ CUtensorMap msrc, const __grid_constant__ CUtensorMap mV,
                  const __grid_constant__ CUtensorMap mdst, const TmaPassArgs a, const TmaBatchArgs ba)
{
    using G = FXy<N, BATCH>;
    constexpr int E = G::E, TT = G::TT, P = G::P, K = G::K, UNIT = G::UNIT, S = G::S;
    constexpr uint32_t kUnitBytes = UNIT * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    float *s_src = reinterpret_cast<float *>(smem_raw + pad);
    float *s_vt = s_src + S * UNIT;
    float *s_mult = s_vt + S * UNIT;  // batched: [S][x row, y row]; single: x row, y row
    float2 *s_tw = reinterpret_cast<float2 *>(s_mult + (BATCH ? S * 2 * N : 2 * N));
    uint64_t *full = reinterpret_cast<uint64_t *>(s_tw + N);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    for (int i = tid; i < N; i += G::THREADS) {
        s_tw[i] = BATCH ? ba.tw[i] : a.tw[i];
        if (!BATCH) {
            s_mult[i] = a.mult[i];
            s_mult[N + i] = a.mult_y[i];
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
    // x mapping: thread tx of line pair lx; y mapping: column pair p, thread ty, plane kk
    const int tx = tid % TT, lx = tid / TT;
    const int p = tid % P, ty = (tid / P) % TT, kk = tid / (P * TT);
    float mrow[E];
#pragma unroll
    for (int e = 0; e < E; ++e) mrow[e] = BATCH ? 0.f : s_mult[tx + e * TT];
    const int fsrc = BATCH ? (ba.src >= 0 ? ba.src : 1 - ba.dst) : 0;

    const int units = BATCH ? ba.tiles : a.n_tiles;
    const int total = BATCH ? ba.members * ba.tiles : a.n_tiles;
    const int nk = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto at = [&](int k, int &i, int &z0) {
        const int g = (int)blockIdx.x + k * (int)gridDim.x;
        i = g / units;
        z0 = (g - i * units) * K;
    };
    auto issue = [&](int k) {
        const int s = k % S;
        int i, z0;
        at(k, i, z0);
        if constexpr (BATCH) {
            const TmaMember *mm = ba.mem + i;
            mbar_arrive_expect_tx(&full[s], 2 * kUnitBytes + 2 * N * sizeof(float));
            tma_load_4d(s_src + s * UNIT, &mm->f[fsrc], 0, 0, 0, z0, &full[s]);
            tma_load_4d_hint(s_vt + s * UNIT, &mm->f[3], 0, 0, 0, z0, &full[s], l2_evict_first_policy());
            bulk_load(s_mult + s * 2 * N, ba.pa[i].mult, N * sizeof(float), &full[s]);
            bulk_load(s_mult + s * 2 * N + N, ba.pa_y[i].mult, N * sizeof(float), &full[s]);
        } else {
            mbar_arrive_expect_tx(&full[s], 2 * kUnitBytes);
            // failure-path test hook, as in the x pass: the launch's first unit may be left unloaded
            if (k == 0 && blockIdx.x == 0 && a.inject && atomicExch(a.inject, 0) != 0) return;
            tma_load_4d(s_src + s * UNIT, &msrc, 0, 0, 0, z0, &full[s]);
            tma_load_4d_hint(s_vt + s * UNIT, &mV, 0, 0, 0, z0, &full[s], l2_evict_first_policy());
        }
    };
    if (tid == 0)
        for (int k = 0; k < S - 1 && k < nk; ++k) issue(k);

    for (int k = 0; k < nk; ++k) {
        const int s = k % S;
        int i, z0;
        at(k, i, z0);
        if (!red_stage_wait(&full[s], (uint32_t)((k / S) & 1))) {
            if (tid == 0) red_timeout_exit<S>(full, k, nk, BATCH ? ba.mem[i].status : a.status);
            return;
        }
        float *src = s_src + s * UNIT;
        float *vt = s_vt + s * UNIT;
        const float *multy = BATCH ? s_mult + s * 2 * N + N : s_mult + N;
        // 1. x elements and the V term into registers
        XTile<N, E> x;
        x.load(src, vt, BATCH ? ba.pa[i].bV : a.bV, true, tx, lx);
        __syncthreads();
        // 2.-3. y lines ([K][N][P] complex pairs) read from src, transformed
        // with the V tile (no longer needed) as exchange space and result
        {
            const int l0 = kk * N * P + p;
            sred_tile<N, E>(reinterpret_cast<const float2 *>(src) + l0, reinterpret_cast<float2 *>(vt) + l0, P, multy,
                            s_tw, ty);
        }
        __syncthreads();
        // 4. x lines, plus the V term and the y result of each element
        if constexpr (BATCH) {
            float mr[E];
#pragma unroll
            for (int e = 0; e < E; ++e) mr[e] = s_mult[s * 2 * N + tx + e * TT];
            x.finish(src, mr, s_tw, vt);
        } else {
            x.finish(src, mrow, s_tw, vt);
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tma_reduce_add_4d(BATCH ? &ba.mem[i].f[ba.dst] : &mdst, 0, 0, 0, z0, src);
            bulk_commit();
            if (k + S - 1 < nk) {
                bulk_wait_read<1>();
                issue(k + S - 1);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace spstd
