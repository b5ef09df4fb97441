// Instantiations and launchers of the four-step long-line x pass (both precisions).
#include "launch.cuh"
#include "longline.h"

namespace spstd {

namespace {

#define SPSTD_N1_CASES(M) M(2) M(4) M(8) M(16) M(32) M(64) M(128) M(256) M(512) M(1024)

template <typename T, int N1>
cudaError_t lcol_n(const LongArgs<T> &a, bool inverse, bool prepare, cudaStream_t s)
{
    constexpr int TT = lcol_tt<T, N1>();
    constexpr int LPC = lcol_lpc<T, N1>();
    constexpr size_t smem = lcol_smem<T, N1>();
    cudaError_t e = inverse ? allow_smem<lcol_inv_kernel<T, N1>>(smem) : allow_smem<lcol_fwd_kernel<T, N1>>(smem);
    if (e != cudaSuccess || prepare) return e;
    if (a.N2 % LPC != 0) return cudaErrorInvalidValue;
    const int64_t blocks = a.n_pairs * (a.N2 / LPC);
    if (blocks <= 0) return cudaSuccess;
    if (inverse)
        lcol_inv_kernel<T, N1><<<(unsigned)blocks, dim3(LPC, TT), smem, s>>>(a);
    else
        lcol_fwd_kernel<T, N1><<<(unsigned)blocks, dim3(LPC, TT), smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N2>
cudaError_t lrow_n(const LongArgs<T> &a, bool prepare, cudaStream_t s)
{
    constexpr int TT = lrow_tt<T, N2>();
    constexpr int LPC = lrow_lpc<T, N2>();
    constexpr size_t smem = lrow_smem<T, N2>();
    cudaError_t e = allow_smem<lrow_kernel<T, N2>>(smem);
    if (e != cudaSuccess || prepare) return e;
    const int64_t rows = a.n_pairs * a.N1;
    const int64_t blocks = (rows + LPC - 1) / LPC;
    if (blocks <= 0) return cudaSuccess;
    lrow_kernel<T, N2><<<(unsigned)blocks, dim3(TT, LPC), smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t lcol_any(const LongArgs<T> &a, bool inverse, bool prepare, cudaStream_t s)
{
    switch (a.N1) {
#define SPSTD_C(n) \
    case n: return lcol_n<T, n>(a, inverse, prepare, s);
        SPSTD_N1_CASES(SPSTD_C)
#undef SPSTD_C
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t lrow_any(const LongArgs<T> &a, bool prepare, cudaStream_t s)
{
    switch (a.N2) {
    case 1024: return lrow_n<T, 1024>(a, prepare, s);
    case 2048: return lrow_n<T, 2048>(a, prepare, s);
    case 4096: return lrow_n<T, 4096>(a, prepare, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_long_x(const LongArgs<T> &a, cudaStream_t s, int which)
{
    cudaError_t e;
    if ((which < 0 || which == 0) && (e = lcol_any<T>(a, false, false, s)) != cudaSuccess) return e;
    if ((which < 0 || which == 1) && (e = lrow_any<T>(a, false, s)) != cudaSuccess) return e;
    if (which < 0 || which == 2) return lcol_any<T>(a, true, false, s);
    return cudaSuccess;
}

template <typename T>
cudaError_t prepare_long_x(int N1, int N2)
{
    LongArgs<T> a{};
    a.N1 = N1;
    a.N2 = N2;
    cudaError_t e;
    if ((e = lcol_any<T>(a, false, true, nullptr)) != cudaSuccess) return e;
    if ((e = lcol_any<T>(a, true, true, nullptr)) != cudaSuccess) return e;
    return lrow_any<T>(a, true, nullptr);
}

template cudaError_t launch_long_x<float>(const LongArgs<float> &, cudaStream_t, int);
template cudaError_t launch_long_x<double>(const LongArgs<double> &, cudaStream_t, int);
template cudaError_t prepare_long_x<float>(int, int);
template cudaError_t prepare_long_x<double>(int, int);

}  // namespace spstd
