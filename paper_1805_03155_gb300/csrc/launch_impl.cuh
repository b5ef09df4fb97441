// launch_impl.cuh -- definitions of Launch<T>; included by exactly one
// translation unit per precision.
#pragma once

#include "launch.cuh"

namespace spstd {

template <typename T>
cudaError_t Launch<T>::xpass(int N, const PassArgs<T> &a, cudaStream_t s)
{
#define SPSTD_X(n) xpass_n<T, n>(a, s)
    switch (N) {
    case 2: return SPSTD_X(2);
    case 4: return SPSTD_X(4);
    case 8: return SPSTD_X(8);
    case 16: return SPSTD_X(16);
    case 32: return SPSTD_X(32);
    case 64: return SPSTD_X(64);
    case 128: return SPSTD_X(128);
    case 256: return SPSTD_X(256);
    case 512: return SPSTD_X(512);
    case 1024: return SPSTD_X(1024);
    case 24: return SPSTD_X(24);
    case 48: return SPSTD_X(48);
    case 96: return SPSTD_X(96);
    case 192: return SPSTD_X(192);
    case 384: return SPSTD_X(384);
    case 2048: return SPSTD_X(2048);
    case 4096: return SPSTD_X(4096);
    case 8192: return SPSTD_X(8192);
    default: return cudaErrorInvalidValue;
    }
#undef SPSTD_X
}

template <typename T>
cudaError_t Launch<T>::spass(int N, const PassArgs<T> &a, cudaStream_t s)
{
#define SPSTD_S(n) spass_n<T, n>(a, s)
    switch (N) {
    case 2: return SPSTD_S(2);
    case 4: return SPSTD_S(4);
    case 8: return SPSTD_S(8);
    case 16: return SPSTD_S(16);
    case 32: return SPSTD_S(32);
    case 64: return SPSTD_S(64);
    case 128: return SPSTD_S(128);
    case 256: return SPSTD_S(256);
    case 512: return SPSTD_S(512);
    case 1024: return SPSTD_S(1024);
    case 24: return SPSTD_S(24);
    case 48: return SPSTD_S(48);
    case 96: return SPSTD_S(96);
    case 192: return SPSTD_S(192);
    case 384: return SPSTD_S(384);
    default: return cudaErrorInvalidValue;
    }
#undef SPSTD_S
}

template <typename T>
int Launch<T>::resident_max_n()
{
    return sizeof(T) == 4 ? 8192 : 4096;
}

template <typename T>
cudaError_t Launch<T>::resident1d(int N, const ResidentArgs<T> &a, cudaStream_t s)
{
#define SPSTD_R(n) resident_n<T, n>(a, s)
    switch (N) {
    case 2: return SPSTD_R(2);
    case 4: return SPSTD_R(4);
    case 8: return SPSTD_R(8);
    case 16: return SPSTD_R(16);
    case 32: return SPSTD_R(32);
    case 64: return SPSTD_R(64);
    case 128: return SPSTD_R(128);
    case 256: return SPSTD_R(256);
    case 512: return SPSTD_R(512);
    case 1024: return SPSTD_R(1024);
    case 2048: return SPSTD_R(2048);
    case 4096: return SPSTD_R(4096);
    default: break;
    }
    if constexpr (sizeof(T) == 4) {
        if (N == 8192) return SPSTD_R(8192);
    }
    return cudaErrorInvalidValue;
#undef SPSTD_R
}

// line lengths of the 2D/3D passes: powers of two and 3 * 2^k (radix-3 first stage)
#define SPSTD_CASES(M)                                                     \
    M(2) M(4) M(8) M(16) M(32) M(64) M(128) M(256) M(512) M(1024)        \
    M(24) M(48) M(96) M(192) M(384)

template <typename T>
int Launch<T>::xpass_tiles(int N, int64_t n_rows)
{
    const int64_t pairs = (n_rows + 1) / 2;
    int lpc = 0;
#define SPSTD_C(n) \
    if (N == n) lpc = xpass_lpc<T, n>();
    SPSTD_CASES(SPSTD_C)
#undef SPSTD_C
    if (N == 2048) lpc = xpass_lpc<T, 2048>();
    if (N == 4096) lpc = xpass_lpc<T, 4096>();
    if (N == 8192) lpc = xpass_lpc<T, 8192>();
    return lpc ? (int)((pairs + lpc - 1) / lpc) : 0;
}

template <typename T>
int Launch<T>::spass_tiles(int N, int nx, int64_t n_outer)
{
    int lpc = 0;
#define SPSTD_C(n) \
    if (N == n) lpc = spass_lpc<T, n>();
    SPSTD_CASES(SPSTD_C)
#undef SPSTD_C
    return lpc ? (int)(((nx + 2 * lpc - 1) / (2 * lpc)) * n_outer) : 0;
}

template <typename T>
cudaError_t Launch<T>::xpass_batch(int N, const PassArgs<T> *args, int members, int tiles, cudaStream_t s)
{
    switch (N) {
#define SPSTD_C(n) \
    case n: return xpass_batch_n<T, n>(args, members, tiles, s);
        SPSTD_CASES(SPSTD_C)
#undef SPSTD_C
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t Launch<T>::spass_batch(int N, const PassArgs<T> *args, int members, int tiles, cudaStream_t s)
{
    switch (N) {
#define SPSTD_C(n) \
    case n: return spass_batch_n<T, n>(args, members, tiles, s);
        SPSTD_CASES(SPSTD_C)
#undef SPSTD_C
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t Launch<T>::resident_batch(int N, const ResidentArgs<T> *args, int members, int64_t nsteps,
                                      cudaStream_t s)
{
    switch (N) {
#define SPSTD_C(n) \
    case n: return resident_batch_n<T, n>(args, members, nsteps, s);
        // 1D grids: power-of-two lengths only
        SPSTD_C(2) SPSTD_C(4) SPSTD_C(8) SPSTD_C(16) SPSTD_C(32) SPSTD_C(64) SPSTD_C(128) SPSTD_C(256)
        SPSTD_C(512) SPSTD_C(1024)
#undef SPSTD_C
    case 2048: return resident_batch_n<T, 2048>(args, members, nsteps, s);
    case 4096: return resident_batch_n<T, 4096>(args, members, nsteps, s);
    default: break;
    }
    if constexpr (sizeof(T) == 4) {
        if (N == 8192) return resident_batch_n<T, 8192>(args, members, nsteps, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::probe_batch(const ProbeMember<T> *members, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    probe_batch_kernel<T><<<count, 32, 0, s>>>(members);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::probe_snapshot(const T *psiR, const T *psiI, const ProbeArgs &a, double2 *snap,
                                      cudaStream_t s)
{
    probe_snapshot_kernel<T><<<1, 32, 0, s>>>(psiR, psiI, a, snap);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::probe_merged(const T *psiR, const T *psiI, const ProbeArgs &a, const double2 *snap,
                                    double alpha, int mf, cudaStream_t s)
{
    probe_merged_kernel<T><<<1, 32, 0, s>>>(psiR, psiI, a, snap, alpha, mf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::eigen_accum(const T *psiR, const T *psiI, double2 *acc, int64_t n, int n_target,
                                   const double *theta, int64_t window, int64_t *step, unsigned *done,
                                   cudaStream_t s)
{
    int64_t b = (n + 255) / 256;
    if (b > 2048) b = 2048;
    if (b < 1) b = 1;
    eigen_accum_kernel<T><<<(unsigned)b, 256, 0, s>>>(psiR, psiI, acc, n, n_target, theta, window, step, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rk4_update(const T *yR, const T *yI, const T *hR, const T *hI, const T *aR, const T *aI,
                                  T *oR, T *oI, T *tR, T *tI, int64_t n, T cb, T ca, int last, cudaStream_t s)
{
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    rk4_update_kernel<T><<<(unsigned)b, 256, 0, s>>>(yR, yI, hR, hI, aR, aI, oR, oI, tR, tI, n, cb, ca, last);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dense_pass(const DenseArgs<T> &a, cudaStream_t s)
{
    if (a.n_lines <= 0) return cudaSuccess;
    const int64_t blocks = (a.n_lines + kDenseLines - 1) / kDenseLines;
    const int threads = (a.n + 31) / 32 * 32;
    const size_t smem = sizeof(T) * (size_t)kDenseLines * a.n;
    dense_pass_kernel<T><<<(unsigned)blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dense_resident1d(const DenseResidentArgs<T> &a, cudaStream_t s)
{
    const int threads = ((a.n > a.n_probe ? a.n : a.n_probe) + 31) / 32 * 32;
    dense_resident1d_kernel<T><<<1, threads, 2 * sizeof(T) * a.n, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::probe(const T *psiR, const T *psiI, const ProbeArgs &a, cudaStream_t s)
{
    probe_kernel<T><<<1, 32, 0, s>>>(psiR, psiI, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dot2(const T *x1, const T *y1, const T *x2, const T *y2, int64_t n, double *partial,
                            int nblocks, cudaStream_t s)
{
    dot2_kernel<T><<<nblocks, 256, 0, s>>>(x1, y1, x2, y2, n, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::from_f64(const double *in, T *out, int64_t n, cudaStream_t s)
{
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    from_f64_kernel<T><<<(unsigned)b, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_f64(const T *in, double *out, int64_t n, cudaStream_t s)
{
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    to_f64_kernel<T><<<(unsigned)b, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace spstd
