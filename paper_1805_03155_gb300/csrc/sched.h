// sched.h -- schedules (radix and tile plans) of the plain pass kernels, the
// choices the autotuner times.  A schedule is chosen per axis:
//   0  the default kernel of the axis (the pipelined TMA pass with its
//      reduce-add epilogue where one exists,
//      else the plain pass with E = 16 FP32 / 8 FP64 points per thread and
//      about 256 threads per block)
//   1  plain, half the lines per block
//   2  plain, twice the lines per block
//   3  plain, half the points per thread (one radix lower per stage), half
//      the lines per block
//   4  plain, the default plan (differs from 0 only on TMA axes); on a dense
//      wall axis whose 0 is the tensor-core pass: the CUDA-core dense pass
//   5  the TMA pass with loaded and stored destination tiles (TMA axes only)
//   6  x axes of 32, 48, 64, 96, 128 or 256 points (FP32 2D/3D grids, single
//      and batched): the reduce-add TMA pass with per-warp tiles
//      (pass_tmared.cuh, xpass_warp_kernel); same bits as 0
// Schedules 1..3 exist for lines of kSchedMinN..kSchedMaxN points; 1, 2 and 4
// run exactly the arithmetic of the default plain kernel (same results bit for
// bit), 3 changes the radix sequence and so the rounding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace spstd {

constexpr int kSchedules = 7;
constexpr int kSchedMinN = 32;
constexpr int kSchedMaxN = 512;

inline bool sched_tunable_n(int64_t N) { return N >= kSchedMinN && N <= kSchedMaxN && (N & (N - 1)) == 0; }

// Whether schedule v (1..3) exists for a pass of this kind (axis 0: x pass,
// else strided) at line length N.
template <typename T>
bool sched_valid(int axis, int N, int v);

// Launchers of schedules 1..3 (same contracts as Launch<T>::xpass / spass and
// their batched forms; a call with no work only raises the shared-memory limit).
template <typename T>
cudaError_t xpass_sched(int N, int v, const PassArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t spass_sched(int N, int v, const PassArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t xpass_batch_sched(int N, int v, const PassArgs<T> *args, int members, int tiles, cudaStream_t s);
template <typename T>
cudaError_t spass_batch_sched(int N, int v, const PassArgs<T> *args, int members, int tiles, cudaStream_t s);
// Blocks one member of a batched pass needs under schedule v.
template <typename T>
int xpass_tiles_sched(int N, int v, int64_t n_rows);
template <typename T>
int spass_tiles_sched(int N, int v, int nx, int64_t n_outer);

}  // namespace spstd
