// launch.cuh -- host-side launchers of the half-stage kernels, instantiated
// once per precision (kernels_f32.cu, kernels_f64.cu).  Each launcher picks
// the compile-time line length N by a switch and sets the block shape:
//   x pass        block (TT, LPC), LPC line pairs per block (~256 threads)
//   strided pass  block (LPC, TT), 2 LPC adjacent x columns per block
//   resident 1D   block (TT), one block per grid
// with TT = N/E threads per line and E elements per thread (16 FP32, 8 FP64).
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace spstd {

template <typename T, int N>
constexpr int threads_per_line() { return N / line_e<T, N>::value; }

template <typename T, int N>
constexpr int xpass_lpc()
{
    return threads_per_line<T, N>() >= 256 ? 1 : 256 / threads_per_line<T, N>();
}

template <typename T, int N>
constexpr int spass_lpc()
{
    constexpr int cap = sizeof(T) == 4 ? 16 : 8;
    constexpr int l = threads_per_line<T, N>() >= 256 ? 1 : 256 / threads_per_line<T, N>();
    return l > cap ? cap : l;
}

// Lets a kernel use more than 48 KB of dynamic shared memory.  The attribute
// is per kernel and per device, so the "done" mask is per instantiation.
template <auto Kernel>
inline cudaError_t allow_smem(size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static unsigned long long done = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}

template <typename T, int N>
cudaError_t xpass_n(const PassArgs<T> &a, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr int LPC = xpass_lpc<T, N>();
    constexpr size_t smem = xpass_smem<T, N, LPC>();
    auto k = xpass_kernel<T, N, LPC>;
    cudaError_t e = allow_smem<xpass_kernel<T, N, LPC>>(smem);
    if (e != cudaSuccess) return e;
    const int64_t pairs = (a.n_rows + 1) / 2;
    const int64_t blocks = (pairs + LPC - 1) / LPC;
    if (blocks <= 0) return cudaSuccess;
    k<<<dim3((unsigned)blocks), dim3(TT, LPC), smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t spass_n(const PassArgs<T> &a, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr int LPC = spass_lpc<T, N>();
    constexpr size_t smem = spass_smem<T, N, LPC>();
    auto k = spass_kernel<T, N, LPC>;
    cudaError_t e = allow_smem<spass_kernel<T, N, LPC>>(smem);
    if (e != cudaSuccess) return e;
    const int64_t n_xt = (a.nx + 2 * LPC - 1) / (2 * LPC);
    const int64_t blocks = n_xt * a.n_outer;
    if (blocks <= 0) return cudaSuccess;
    k<<<dim3((unsigned)blocks), dim3(LPC, TT), smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t resident_n(const ResidentArgs<T> &a, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr size_t smem = resident_smem<T, N>();
    auto k = resident1d_kernel<T, N>;
    cudaError_t e = allow_smem<resident1d_kernel<T, N>>(smem);
    if (e != cudaSuccess) return e;
    k<<<1, TT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *partial, int count, double *out, cudaStream_t s);

template <typename T, int N>
cudaError_t xpass_batch_n(const PassArgs<T> *args, int members, int tiles, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr int LPC = xpass_lpc<T, N>();
    constexpr size_t smem = xpass_smem<T, N, LPC>();
    cudaError_t e = allow_smem<xpass_batch_kernel<T, N, LPC>>(smem);
    if (e != cudaSuccess || members <= 0 || tiles <= 0) return e;
    xpass_batch_kernel<T, N, LPC><<<dim3((unsigned)(members * tiles)), dim3(TT, LPC), smem, s>>>(args, tiles);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t spass_batch_n(const PassArgs<T> *args, int members, int tiles, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr int LPC = spass_lpc<T, N>();
    constexpr size_t smem = spass_smem<T, N, LPC>();
    cudaError_t e = allow_smem<spass_batch_kernel<T, N, LPC>>(smem);
    if (e != cudaSuccess || members <= 0 || tiles <= 0) return e;
    spass_batch_kernel<T, N, LPC><<<dim3((unsigned)(members * tiles)), dim3(LPC, TT), smem, s>>>(args, tiles);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t resident_batch_n(const ResidentArgs<T> *args, int members, int64_t nsteps, cudaStream_t s)
{
    constexpr int TT = threads_per_line<T, N>();
    constexpr size_t smem = resident_smem<T, N>();
    cudaError_t e = allow_smem<resident1d_batch_kernel<T, N>>(smem);
    if (e != cudaSuccess || members <= 0) return e;
    resident1d_batch_kernel<T, N><<<members, TT, smem, s>>>(args, nsteps);
    return cudaGetLastError();
}

template <typename T> struct Launch {
    static cudaError_t xpass(int N, const PassArgs<T> &a, cudaStream_t s);
    static cudaError_t spass(int N, const PassArgs<T> &a, cudaStream_t s);
    static cudaError_t resident1d(int N, const ResidentArgs<T> &a, cudaStream_t s);
    static cudaError_t probe(const T *psiR, const T *psiI, const ProbeArgs &a, cudaStream_t s);
    static cudaError_t dot2(const T *x1, const T *y1, const T *x2, const T *y2, int64_t n,
                            double *partial, int nblocks, cudaStream_t s);
    static cudaError_t from_f64(const double *in, T *out, int64_t n, cudaStream_t s);
    static cudaError_t to_f64(const T *in, double *out, int64_t n, cudaStream_t s);
    static int resident_max_n();
    // blocks one member of a batched pass needs
    static int xpass_tiles(int N, int64_t n_rows);
    static int spass_tiles(int N, int nx, int64_t n_outer);
    // batched launches over members of one shape (args: device arrays)
    static cudaError_t xpass_batch(int N, const PassArgs<T> *args, int members, int tiles, cudaStream_t s);
    static cudaError_t spass_batch(int N, const PassArgs<T> *args, int members, int tiles, cudaStream_t s);
    static cudaError_t resident_batch(int N, const ResidentArgs<T> *args, int members, int64_t nsteps,
                                      cudaStream_t s);
    static cudaError_t probe_batch(const ProbeMember<T> *members, int count, cudaStream_t s);
    static cudaError_t dense_pass(const DenseArgs<T> &a, cudaStream_t s);
    static cudaError_t rk4_update(const T *yR, const T *yI, const T *hR, const T *hI, const T *aR, const T *aI,
                                  T *oR, T *oI, T *tR, T *tI, int64_t n, T cb, T ca, int last, cudaStream_t s);
    static cudaError_t eigen_accum(const T *psiR, const T *psiI, double2 *acc, int64_t n, int n_target,
                                   const double *theta, int64_t window, int64_t *step, unsigned *done,
                                   cudaStream_t s);
    static cudaError_t probe_snapshot(const T *psiR, const T *psiI, const ProbeArgs &a, double2 *snap,
                                      cudaStream_t s);
    static cudaError_t probe_merged(const T *psiR, const T *psiI, const ProbeArgs &a, const double2 *snap,
                                    double alpha, int mf, cudaStream_t s);
    static cudaError_t dense_resident1d(const DenseResidentArgs<T> &a, cudaStream_t s);
};

}  // namespace spstd
