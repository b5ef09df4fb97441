// pass_tma_launch.h -- host interface of the pipelined FP32 passes.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

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
};

// Tile geometry the tensor maps must use.
constexpr unsigned tma_rows_per_tile() { return 32; }  // x pass: contiguous rows per tile
constexpr unsigned tma_cols_per_tile() { return 32; }  // strided pass: x columns per tile

// axis 0: x pass, 1: y pass, 2: z pass; N in {64, 128, 256}.  Raises the
// kernel's shared-memory limit and sizes the persistent grid on first use.
cudaError_t launch_pass_tma(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mdst,
                            const TmaPassArgs &a, cudaStream_t s);
// The same set-up without a launch (call before a stream capture).
cudaError_t prepare_pass_tma(int axis, int N);

// Reduce-add variants (the dst tile is accumulated by a TMA reduce at L2
// instead of being loaded and stored): mV is the potential in the x view
// (x pass only; unused otherwise).
cudaError_t launch_pass_tmared(int axis, int N, const CUtensorMap &msrc, const CUtensorMap &mV,
                               const CUtensorMap &mdst, const TmaPassArgs &a, cudaStream_t s);
cudaError_t prepare_pass_tmared(int axis, int N);
// Rows per tile of the reduce-add x pass (its x-view maps use this box height).
int tmared_x_rows();

struct XyPassArgs;
// x and y passes of a 3D half-stage in one persistent launch (pass_xy.cuh);
// nx = ny = N in {64, 128, 256}; maps: src and dst in the x view (N x 32-row
// box) and the y view (32-column x N box).
cudaError_t launch_xypass_tma(int N, const CUtensorMap &src_x, const CUtensorMap &dst_x, const CUtensorMap &src_y,
                              const CUtensorMap &dst_y, const XyPassArgs &a, cudaStream_t s);
cudaError_t prepare_xypass_tma(int N);

}  // namespace spstd
