// dense_tc.h -- the dense spectral operator of a wall axis (Section 2.2: the
// DST / DCT second derivative, or a short periodic axis) applied on the
// tensor cores: for every line of the axis, dst += a (D src) (+ bV V src on
// the x axis), D the n x n operator times hbar/2m*.  Over all lines of an
// axis this is one dense product Y = X D^T (X: lines x n), run as tcgen05
// TF32 MMAs with FP32 accumulation in tensor memory.  FP32 accuracy comes
// from the 3xTF32 split: D = D_hi + D_lo (split in FP64 on the host), X =
// X_hi + X_lo (split in the kernel), and X D^T ~ X_hi D_hi^T + X_hi D_lo^T +
// X_lo D_hi^T (the dropped X_lo D_lo^T term is ~2^-22 relative).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spstd {

// Lines of 32..128 points (FP32 2D/3D grids): the operator pair (128 KB at
// n = 128) stays in shared memory for the whole launch.
constexpr int kDenseTcMinN = 32;
constexpr int kDenseTcMaxN = 128;
inline bool dense_tc_eligible(int64_t n) { return n >= kDenseTcMinN && n <= kDenseTcMaxN; }
// n padded to the MMA's K and N granule (a multiple of 32).
inline int dense_tc_pad(int64_t n) { return (int)((n + 31) / 32 * 32); }
// Float index of operator element (i, j) in the K-major, unswizzled operand
// layout: core matrices of 8 rows x 4 values (128 contiguous bytes), adjacent
// along j 128 bytes apart, 8-row groups np/4 core matrices apart.
inline size_t dense_tc_offset(int i, int j, int np)
{
    return ((size_t)(i >> 3) * (size_t)(np / 4) * 128 + (size_t)(j >> 2) * 128 + (size_t)(i & 7) * 16 +
            (size_t)(j & 3) * 4) / 4;
}

struct DenseTcArgs {
    const float *src;
    float *dst;
    const float *V;           // x axis: the potential (use_V)
    // hbar/2m* D(i, j) (i output point, j input point; zero padded to np x np),
    // split as hi + lo, each np*np floats in the MMA's shared-memory layout:
    // element (i, j) at dense_tc_offset(i, j, np)
    const float *Dhi, *Dlo;
    float a, bV;
    int use_V;
    int n, np;                // points per line; n padded to a multiple of 32
    int64_t stride;           // elements between consecutive points of a line
    int64_t inner, outer_stride, n_lines;  // line l starts at (l / inner) outer_stride + (l % inner)
    int *status;              // device status word (kStatusTimeout on a timed-out wait)
};

// Launches the pass (persistent grid, one 256-thread block per SM); with
// a.src == nullptr it only raises the kernel's shared-memory limit.
cudaError_t launch_dense_tc(const DenseTcArgs &a, cudaStream_t s);

}  // namespace spstd
