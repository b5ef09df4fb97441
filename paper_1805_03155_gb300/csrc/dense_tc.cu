// dense_tc.cu -- the dense wall pass on the tensor cores (dense_tc.h): tcgen05
// TF32 MMAs (cta_group::1, M = 128 lines, N = K = n padded to 32) with the
// accumulator in tensor memory, the 3xTF32 split for FP32 accuracy.
//
// One persistent 256-thread block per SM keeps the operator pair D_hi, D_lo
// in shared memory (the B operand, K-major: row i of D holds the inputs j of
// output point i; two bulk copies of tables already in that layout) and walks
// tiles of 128 lines.  Per tile, chunks of 32 input points are staged as
// X_hi / X_lo (the A operand, K-major: one row per line) by all threads from
// registers loaded one chunk ahead; thread 0 issues the chunk's MMAs (X_hi
// D_hi, X_hi D_lo, X_lo D_hi for each K step of 8) and commits them to an
// mbarrier; the next chunk's loads run while the MMAs do, then the block waits
// (bounded) before the chunk's buffers are refilled.  After the last chunk
// every warp reads its 32 lines x half the output points from tensor memory
// (tcgen05.ld) and adds a (D src) (+ bV V src on the x axis) to dst.  A wait
// that runs out records kStatusTimeout, waits once more (bounded) for the
// copies and MMAs in flight, frees the tensor memory and returns.
#include "dense_tc.h"
#include "persist.cuh"
#include "tma.cuh"

namespace spstd {
namespace {

constexpr int kTcM = 128;        // lines per tile: the MMA's M (one tensor-memory lane each)
constexpr int kTcK = 32;         // input points per staged chunk
constexpr int kTcThreads = 256;  // 8 warps: 4 lane quarters x 2 column halves in the epilogue
constexpr uint32_t kCoreBytes = 128;  // one core matrix: 8 rows x 16 bytes

// Byte offset of element (row, k) of a K-major operand without swizzle: core
// matrices of 8 rows x 4 TF32 values (16 bytes a row), 128 contiguous bytes
// each; consecutive core matrices along K are kCoreBytes apart (the
// descriptor's leading byte offset), consecutive 8-row groups sbo bytes apart
// (its stride byte offset).
__device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * kCoreBytes + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets in 16-byte units (bits 0-13, 16-29, 32-45), descriptor version 1
// (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1),
// A and B TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// x rounded to TF32 (10 mantissa bits, to nearest, ties away from zero).
__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// D[tmem] (+)= A B, A and B from shared memory; accumulate != 0 adds to D.
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One arrival on bar once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 columns of 32-bit values from tensor memory: thread t of the
// warp gets lane (taddr lane + t), columns taddr column .. + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tmem_cols(int nc) { return nc <= 32 ? 32u : nc <= 64 ? 64u : 128u; }

// Output points may be split over dense_tc_split(np) blocks per tile (N = np
// / split each), each keeping only its rows of D.  Measured at 128^3 walls:
// two blocks per tile (two per SM) took 38.6 us per pass against 26.5 us for
// one (each tile's chunks are then staged twice), so the split is 1.
__host__ __device__ __forceinline__ int dense_tc_split(int) { return 1; }

// This thread's 16 elements of the A chunk (lines l0 .., inputs kc*32 ..;
// zero past the grid), in the order of a_slot: element r sits at row
// m = ((w + 8r) mod 16) 8 + (lane mod 8), input k = ((w + 8r) / 16) 4 +
// lane / 8, so the 32 lanes of a warp store to distinct banks.
__device__ __forceinline__ void a_rc(int r, int warp, int lane, int &m, int &k)
{
    const int blk = warp + 8 * r;
    m = (blk & (kTcM / 8 - 1)) * 8 + (lane & 7);
    k = (blk / (kTcM / 8)) * 4 + (lane >> 3);
}

// With warp < 8, element r's row is (warp + 8 (r mod 2)) 8 + lane mod 8: a
// thread's 16 elements lie on two lines, whose first points (or -1 past the
// grid) are found once per tile.
__device__ __forceinline__ void line_bases(const DenseTcArgs &a, int64_t l0, int warp, int lane, int64_t (&b)[2])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t line = l0 + (warp + 8 * h) * 8 + (lane & 7);
        b[h] = line < a.n_lines ? (line / a.inner) * a.outer_stride + (line % a.inner) : -1;
    }
}

__device__ __forceinline__ void load_chunk(const DenseTcArgs &a, const int64_t (&b)[2], int kc, int lane,
                                           float (&v)[16])
{
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int j = kc * kTcK + (r >> 1) * 4 + (lane >> 3);  // a_rc's k
        const int64_t lb = b[r & 1];
        v[r] = (lb >= 0 && j < a.n) ? __ldg(a.src + lb + (int64_t)j * a.stride) : 0.f;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) dense_tc_kernel(const DenseTcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    unsigned char *base = smem_raw + pad;
    const int np = a.np;
    const int split = dense_tc_split(np), nc = np / split, part = (int)blockIdx.x % split;
    const uint32_t bbytes = (uint32_t)nc * (uint32_t)np * 4u;  // this block's rows of D
    unsigned char *b_hi = base, *b_lo = base + bbytes;
    unsigned char *a_hi = base + 2 * bbytes, *a_lo = a_hi + kTcM * kTcK * 4;
    uint64_t *bar = reinterpret_cast<uint64_t *>(a_lo + kTcM * kTcK * 4);  // MMA completion
    uint64_t *bbar = bar + 1;                                              // operator copy
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = tmem_cols(nc);
    const uint32_t sbo_b = (uint32_t)(np / 4) * kCoreBytes;   // a B row group spans all np inputs
    const uint32_t sbo_a = (uint32_t)(kTcK / 4) * kCoreBytes;  // an A row group spans one chunk
    const int64_t tiles = (a.n_lines + kTcM - 1) / kTcM;
    const int nchunks = np / kTcK;

    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bbar, 1);
        mbar_fence_init();
        // this block's rows part*nc .. of the operator pair, stored in the B
        // layout already (8-row groups are contiguous): two bulk copies
        mbar_arrive_expect_tx(bbar, 2 * bbytes);
        bulk_load(b_hi, a.Dhi + (size_t)part * nc * np, bbytes, bbar);
        bulk_load(b_lo, a.Dlo + (size_t)part * nc * np, bbytes, bbar);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the first chunk's loads run while the operator arrives
    float v[16];
    const int64_t tstep = gridDim.x / split;
    int64_t tile = blockIdx.x / split;
    int64_t lbase[2], nbase[2] = {-1, -1};
    line_bases(a, tile * kTcM, warp, lane, lbase);
    if (tile < tiles) load_chunk(a, lbase, 0, lane, v);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tf32_idesc(kTcM, nc);
    bool ok = !__syncthreads_or(!mbar_wait(bbar, 0));
    uint32_t phase = 0;
    bool mma_pending = false;  // a chunk's MMAs whose completion wait ran out
    for (; tile < tiles && ok; tile += tstep) {
        const int64_t l0 = tile * kTcM;
        for (int kc = 0; kc < nchunks; ++kc) {
            // the chunk into the A layout, split hi + lo
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                int m, k;
                a_rc(r, warp, lane, m, k);
                const float hi = tf32_round(v[r]);
                const uint32_t off = core_off(m, k, sbo_a);
                *reinterpret_cast<float *>(a_hi + off) = hi;
                *reinterpret_cast<float *>(a_lo + off) = tf32_round(v[r] - hi);
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
                for (int kk = 0; kk < kTcK / 8; ++kk) {
                    // K step of 8 inputs: two core matrices along K
                    const uint32_t ao = (uint32_t)kk * 2 * kCoreBytes;
                    const uint32_t bo = (uint32_t)(kc * (kTcK / 8) + kk) * 2 * kCoreBytes;
                    const uint64_t dah = smem_desc(ah + ao, kCoreBytes, sbo_a), dal = smem_desc(al + ao, kCoreBytes, sbo_a);
                    const uint64_t dbh = smem_desc(bh + bo, kCoreBytes, sbo_b), dbl = smem_desc(bl + bo, kCoreBytes, sbo_b);
                    mma_tf32(tmem, dah, dbh, idesc, (kc | kk) != 0);
                    mma_tf32(tmem, dah, dbl, idesc, 1u);
                    mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
                mma_commit(bar);
            }
            // the next chunk's loads (this tile's, or the next tile's first) run with the MMAs
            if (kc + 1 < nchunks) {
                load_chunk(a, lbase, kc + 1, lane, v);
            } else if (tile + tstep < tiles) {
                line_bases(a, (tile + tstep) * kTcM, warp, lane, nbase);
                load_chunk(a, nbase, 0, lane, v);
            }
            // the MMAs must have read the chunk before it is refilled (and,
            // after the last chunk, have written the accumulator)
            const bool done = mbar_wait(bar, phase);
            ok = !__syncthreads_or(!done);
            if (!ok) {
                mma_pending = true;
                break;
            }
            phase ^= 1u;
        }
        if (!ok) break;
        tc_fence_after();
        // epilogue: warp w reads tensor-memory lanes 32 (w mod 4) .. + 31 (its
        // lines) and one of two column ranges (16-column groups) of the block's nc
        const int q = warp & 3, lo_cols = (nc / 16 + 1) / 2 * 16;
        const int cbeg = warp < 4 ? 0 : lo_cols, cend = warp < 4 ? lo_cols : nc;
        const int i0 = part * nc;  // the block's first output point
        const int64_t line = l0 + q * 32 + lane;
        const bool live = line < a.n_lines;
        const int64_t lb = live ? (line / a.inner) * a.outer_stride + (line % a.inner) : 0;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float r[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
            // eight columns at a time: every load first, then the updates (as
            // the CUDA-core pass rounds them: dst + a acc, then + bV V src in
            // one fma)
#pragma unroll
            for (int g = 0; g < 16; g += 8) {
                float d[8], vv[8], ss[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const bool in = live && i0 + c0 + g + c < a.n;
                    const int64_t off = lb + (int64_t)(i0 + c0 + g + c) * a.stride;
                    d[c] = in ? a.dst[off] : 0.f;
                    vv[c] = in && a.use_V ? __ldg(a.V + off) : 0.f;
                    ss[c] = in && a.use_V ? __ldg(a.src + off) : 0.f;
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (live && i0 + c0 + g + c < a.n) {
                        const int64_t off = lb + (int64_t)(i0 + c0 + g + c) * a.stride;
                        const float u = d[c] + a.a * r[g + c];
                        a.dst[off] = a.use_V ? fmaf(a.bV * vv[c], ss[c], u) : u;
                    }
                }
            }
        }
        // every warp has read the accumulator before the next tile's MMAs
        tc_fence_before();
        __syncthreads();
        lbase[0] = nbase[0];
        lbase[1] = nbase[1];
    }
    if (!ok) {
        if (tid == 0) atomicExch(a.status, kStatusTimeout);
        // the operator copy and the MMAs of the chunk whose wait ran out may
        // still run: wait for them once more (bounded) before their shared and
        // tensor memory is given up
        mbar_wait(bbar, 0);
        if (mma_pending) mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace

cudaError_t launch_dense_tc(const DenseTcArgs &a, cudaStream_t s)
{
    // the shared-memory limit and grid are set for the largest operator
    constexpr size_t kMaxSmem = 2ull * kDenseTcMaxN * kDenseTcMaxN * 4 + 2ull * kTcM * kTcK * 4 + 24 + 1024;
    int grid = 0;
    cudaError_t e = persistent_grid<dense_tc_kernel>(kTcThreads, kMaxSmem, &grid);
    if (e != cudaSuccess || !a.src) return e;
    if (a.np % kTcK || a.np < kDenseTcMinN || a.np > kDenseTcMaxN || a.n > a.np || a.n < 1)
        return cudaErrorInvalidValue;
    const int split = dense_tc_split(a.np);
    const int64_t items = (a.n_lines + kTcM - 1) / kTcM * split;  // (tile, output part) pairs
    if (items < grid) grid = (int)items;
    grid -= grid % split;  // block b takes part b mod split of tiles b / split, + grid / split, ...
    if (grid <= 0) return cudaSuccess;
    const size_t smem = 2ull * (a.np / split) * a.np * 4 + 2ull * kTcM * kTcK * 4 + 24 + 1024;
    dense_tc_kernel<<<grid, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace spstd
