// pass_tma_launch.h -- host interface of the pipelined FP32 passes.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace spstd {

struct TmaPassArgs {
    const float2 *tw;    // W_N[k]
    const float *mult;   // a k^2(n)/N
    const float *V;      // x pass: potential (use_V)
    float bV;
    int use_V;
    int rows;            // x pass: number of contiguous lines (n1 n2)
    int n_tiles;
    int n_xt;            // strided pass: tiles across x
    int axis;            // strided pass: 1 (y) or 2 (z)
    int reverse;
    int *status;         // device status word (kStatusTimeout on a timed-out wait)
    int nx;              // reduce-add passes: points along x
    int planes;          // reduce-add strided pass: tmared_planes()
    int *inject;         // reduce-add x pass: when *inject != 0, clears it and leaves the first tile unloaded
    const float *mult_y; // fused x-y pass: the y axis's multipliers (mult: the x axis's)
    // Reduce-add x pass with a separable potential V(x, y, z) = vx(x) + vyz(y, z):
    // the V term is rebuilt from these tables (vx: nx floats; vyz: one float per
    // x line, padded with zeros to a whole number of tiles) instead of read
    // from the V field.  Null: the V field is used.
    const float *vx, *vyz;
};

// Tile geometry the tensor maps must use.
constexpr unsigned tma_rows_per_tile() { return 32; }  // x pass: contiguous rows per tile
constexpr unsigned tma_cols_per_tile() { return 32; }  // strided pass: x columns per tile

// Stored-tile passes (pass_tma.cuh, schedule 5).  axis 0: x pass, 1: y pass,
// 2: z pass; N in {64, 128, 256}.  Raises the kernel's shared-memory limit and
// sizes the persistent grid on first use.
cudaError_t launch_pass_tma(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s);
// The same set-up without a launch (call before a stream capture).
cudaError_t prepare_pass_tma(int axis, int N);

// ---------------------------------------------------------------------------
// Reduce-add passes (pass_tmared.cuh), the default for FP32 lines of 32..512
// points and of 48 and 96 points (3 * 2^k: a radix-3 first stage): the
// destination is accumulated at L2 by a TMA reduce-add.
// ---------------------------------------------------------------------------
constexpr bool tmared_eligible(int64_t N)
{
    return N == 32 || N == 64 || N == 128 || N == 256 || N == 512 || N == 48 || N == 96;
}
// Complex points per thread: 16, or 12 for N = 3 * 2^k.
constexpr int tmared_e(int N) { return N % 3 ? 16 : 12; }
// Floats of one x tile or strided tile part: 4096 (16 KB) for power-of-two
// lines, 3072 (12 KB) for 3 * 2^k lines, so that an x block has 128 threads
// and a strided block of K planes 256.
constexpr int tmared_unit(int N) { return N % 3 ? 4096 : 3072; }
// x pass: rows per tile (the box height of its x-view maps).
constexpr int tmared_rows_x(int N) { return tmared_unit(N) / N; }
// Strided pass over N points along y or z with nx points along x: column
// pairs per tile, at most 64 (its y/z-view maps' box is 2P columns wide) and
// at least 8; the largest such P whose 2P columns divide nx, else the largest
// with 2P <= nx (the last tile across x then runs past the grid: its loads
// read zeros there and its reduce-add skips those columns); 0 if nx < 16.
constexpr int tmared_pairs(int N, int64_t nx)
{
    int P = tmared_unit(N) / N < 64 ? tmared_unit(N) / N : 64;
    while (P > 8 && 2 * (int64_t)P > nx) P /= 2;
    int Q = P;
    while (Q > 8 && nx % (2 * Q) != 0) Q /= 2;
    if (nx % (2 * Q) == 0) P = Q;
    return nx >= 16 ? P : 0;
}
// Strided pass: planes of the outer axis per tile -- enough for 256 threads
// per block (tmared_max_planes), or 1 when the outer axis is shorter than that.
constexpr int tmared_max_planes(int N, int P)
{
    return P > 0 && 256 / (P * (N / tmared_e(N))) > 1 ? 256 / (P * (N / tmared_e(N))) : 1;
}
constexpr int tmared_planes(int N, int P, int64_t outer)
{
    return outer >= tmared_max_planes(N, P) ? tmared_max_planes(N, P) : 1;
}
// Tiles of one grid (or one batch member) shaped n[3] in the pass of axis ax;
// *n_xt: tiles across x (strided passes).
inline int tmared_tiles(int axis, const int64_t *n, int *n_xt)
{
    if (axis == 0) {
        if (n_xt) *n_xt = 1;
        const int R = tmared_rows_x((int)n[0]);
        return (int)((n[1] * n[2] + R - 1) / R);
    }
    const int P = tmared_pairs((int)n[axis], n[0]);
    const int64_t outer = axis == 1 ? n[2] : n[1];
    const int K = tmared_planes((int)n[axis], P, outer);
    const int nxt = P ? (int)((n[0] + 2 * P - 1) / (2 * P)) : 0;
    if (n_xt) *n_xt = nxt;
    return nxt * (int)((outer + K - 1) / K);
}

// Single grid: a.n_tiles / a.n_xt from tmared_tiles, a.nx = points along x,
// a.planes from tmared_planes; mV is the potential in the x view (x pass only).
cudaError_t launch_pass_tmared(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mV,
                               const CUtensorMap &mdst, const TmaPassArgs &a, cudaStream_t s);
// Raises the kernel's shared-memory limit and sizes its persistent grid (call
// before a stream capture); nx: points along x.
cudaError_t prepare_pass_tmared(int axis, int N, int64_t nx, int planes);

// x pass with per-warp tiles (schedule 6): lines of N in {32, 48, 64, 96,
// 128, 256} points (a line's N/E threads, E = 16 or 12 for 3 * 2^k, share a
// warp with the other line pairs of its tile), tiles of xwarp_rows(N) rows (the
// box height of its maps).  Single grid: a.n_tiles = ceil(rows /
// xwarp_rows(N)); the table form is taken when a.vyz is set.
constexpr bool xwarp_eligible(int64_t N)
{
    return N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 256;
}
constexpr int xwarp_rows(int N) { return 2 * (32 / (N / (N % 3 ? 16 : 12))); }
cudaError_t launch_pass_xwarp(int N, const CUtensorMap &msrc, const CUtensorMap &mV, const CUtensorMap &mdst,
                              const TmaPassArgs &a, cudaStream_t s);
cudaError_t prepare_pass_xwarp(int N);

// One member of a batched pass: tensor maps over its own fields (0 psi_R,
// 1 psi_I, 2 scratch; index 3 of the x view is V) with the reduce-add boxes,
// and its device status word.  Lives in device memory (64-byte aligned).
struct TmaMember {
    CUtensorMap x[4];  // x view, box N x tmared_rows_x(N)
    CUtensorMap xw[4]; // x view, box N x xwarp_rows(N) (per-warp x tiles; xwarp_eligible lines)
    CUtensorMap y[3];  // y view, box 2P columns x N
    CUtensorMap z[3];  // z view, box 2P columns x 1 x N
    CUtensorMap f[4];  // fused x-y view (fxy_eligible grids), box N x N x fxy_planes(N)
    int *status;
};

// A batched reduce-add pass over `members` members of one shape: member i
// reads field src (1 - dst when src < 0) through mem[i] and accumulates into
// field dst, with the multipliers pa[i].mult (N floats, 16-byte aligned) and,
// on the x pass, pa[i].bV.  tiles / n_xt from tmared_tiles.
struct TmaBatchArgs {
    const TmaMember *mem;
    const PassArgs<float> *pa;
    const PassArgs<float> *pa_y;  // fused x-y pass: the members' y-axis descriptors (pa: x axis)
    const float2 *tw;  // W_N, the same for every member
    int src, dst;
    int members;
    int tiles;
    int n_xt;
    int nx;            // points along x
    int planes;        // strided pass: tmared_planes()
    int axis;
    int vsep;          // x pass: every member has separable-potential tables (pa[i].vx, pa[i].vyz)
};

cudaError_t launch_pass_tmared_batch(int axis, int N, const TmaBatchArgs &a, cudaStream_t s);
// Batched x pass with per-warp tiles (batch schedule 6; xwarp_eligible lines):
// the members' xw maps, a.tiles = ceil(rows / xwarp_rows(N)) per member; the
// table form when a.vsep.
cudaError_t launch_pass_xwarp_batch(int N, const TmaBatchArgs &a, cudaStream_t s);
cudaError_t prepare_pass_xwarp_batch(int N);

// V[r nx + i] = vx[i] + vyz[r] in FP32 (rounded to nearest), the values the x
// pass rebuilds from the tables of a separable potential; rows = ny nz.
cudaError_t build_separable_v(const float *vx, const float *vyz, float *V, int64_t nx, int64_t rows,
                              cudaStream_t s);

// ---------------------------------------------------------------------------
// Fused x + y reduce-add pass (pass_tmared.cuh) for grids with nx = ny = N in
// {32, 64}: units of fxy_planes(N) planes hold whole x and y lines.  The map
// views the field as (x, y, 1, z) with box (N, N, 1, fxy_planes(N)).
// (96-point planes -- one 36 KB plane per unit, one block per SM -- were
// measured slower than the separate passes on the 512-solve mix.)
// ---------------------------------------------------------------------------
constexpr int fxy_planes(int N) { return 4096 / (N * N); }
inline bool fxy_eligible(const int64_t *n, int dims)
{
    return dims >= 2 && n[0] == n[1] && (n[0] == 32 || n[0] == 64) && (dims == 3 || fxy_planes((int)n[0]) == 1);
}
inline int fxy_units(const int64_t *n) { return (int)((n[2] + fxy_planes((int)n[0]) - 1) / fxy_planes((int)n[0])); }
// Single grid: a.mult / a.mult_y the x and y multipliers, a.n_tiles = fxy_units.
cudaError_t launch_pass_fxy(int N, const CUtensorMap &msrc, const CUtensorMap &mV, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s);
// Batched: a.tiles = fxy_units, a.pa / a.pa_y the x and y descriptors.
cudaError_t launch_pass_fxy_batch(int N, const TmaBatchArgs &a, cudaStream_t s);
cudaError_t prepare_pass_fxy(int N, bool batch);
cudaError_t prepare_pass_tmared_batch(int axis, int N, int64_t nx, int planes);

struct XyPassArgs;
// x and y passes of a 3D half-stage in one persistent launch (pass_xy.cuh);
// nx = ny = N in {64, 128, 256}; maps: src and dst in the x view (N x 32-row
// box) and the y view (32-column x N box).
cudaError_t launch_xypass_tma(int N, const CUtensorMap &src_x, const CUtensorMap &dst_x, const CUtensorMap &src_y,
                              const CUtensorMap &dst_y, const XyPassArgs &a, cudaStream_t s);
cudaError_t prepare_xypass_tma(int N);

}  // namespace spstd
