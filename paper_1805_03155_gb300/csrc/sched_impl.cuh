// sched_impl.cuh -- the schedule variants of the plain pass kernels; included
// by one translation unit per precision and pass kind (SPSTD_SCHED_T, SPSTD_SCHED_X).
#pragma once

#include "launch.cuh"
#include "sched.h"

namespace spstd {

template <typename T, int N, int V, bool X>
struct Plan {
    static constexpr int E0 = line_e<T, N>::value;
    static constexpr int L0 = X ? xpass_lpc<T, N>() : spass_lpc<T, N>();
    static constexpr int E = V == 3 ? E0 / 2 : E0;
    static constexpr int LPC = V == 2 ? 2 * L0 : ((V == 1 || V == 3) ? (L0 / 2 > 0 ? L0 / 2 : 1) : L0);
    static constexpr int TT = N / (E > 0 ? E : 1);
    static constexpr size_t smem = X ? xpass_smem<T, N, LPC>() : spass_smem<T, N, LPC>();
    static constexpr bool valid = V >= 1 && V <= 3 && E >= 2 && TT * LPC <= 1024 && TT * LPC >= 32 &&
                                  smem <= 227 * 1024 && !(V == 1 && L0 < 2);
};

template <typename T, int N, int V, bool X>
cudaError_t plan_launch(const PassArgs<T> *single, const PassArgs<T> *batch, int members, int tiles, cudaStream_t s)
{
    using P = Plan<T, N, V, X>;
    if constexpr (!P::valid) {
        return cudaErrorInvalidValue;
    } else {
        constexpr int E = P::E, LPC = P::LPC, TT = P::TT;
        constexpr size_t smem = P::smem;
        cudaError_t e;
        if (single) {
            if constexpr (X) {
                if ((e = allow_smem<xpass_kernel<T, N, LPC, E>>(smem)) != cudaSuccess) return e;
                const int64_t blocks = ((single->n_rows + 1) / 2 + LPC - 1) / LPC;
                if (blocks <= 0) return cudaSuccess;
                xpass_kernel<T, N, LPC, E><<<(unsigned)blocks, dim3(TT, LPC), smem, s>>>(*single);
            } else {
                if ((e = allow_smem<spass_kernel<T, N, LPC, E>>(smem)) != cudaSuccess) return e;
                const int64_t blocks = (int64_t)((single->nx + 2 * LPC - 1) / (2 * LPC)) * single->n_outer;
                if (blocks <= 0) return cudaSuccess;
                spass_kernel<T, N, LPC, E><<<(unsigned)blocks, dim3(LPC, TT), smem, s>>>(*single);
            }
        } else {
            if constexpr (X) {
                if ((e = allow_smem<xpass_batch_kernel<T, N, LPC, E>>(smem)) != cudaSuccess) return e;
                if (members <= 0 || tiles <= 0) return cudaSuccess;
                xpass_batch_kernel<T, N, LPC, E><<<(unsigned)(members * tiles), dim3(TT, LPC), smem, s>>>(batch, tiles);
            } else {
                if ((e = allow_smem<spass_batch_kernel<T, N, LPC, E>>(smem)) != cudaSuccess) return e;
                if (members <= 0 || tiles <= 0) return cudaSuccess;
                spass_batch_kernel<T, N, LPC, E><<<(unsigned)(members * tiles), dim3(LPC, TT), smem, s>>>(batch, tiles);
            }
        }
        return cudaGetLastError();
    }
}

template <typename T, int N, bool X>
cudaError_t plan_any_v(int v, const PassArgs<T> *single, const PassArgs<T> *batch, int members, int tiles,
                       cudaStream_t s)
{
    switch (v) {
    case 1: return plan_launch<T, N, 1, X>(single, batch, members, tiles, s);
    case 2: return plan_launch<T, N, 2, X>(single, batch, members, tiles, s);
    case 3: return plan_launch<T, N, 3, X>(single, batch, members, tiles, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool X>
cudaError_t plan_any(int N, int v, const PassArgs<T> *single, const PassArgs<T> *batch, int members, int tiles,
                     cudaStream_t s)
{
    switch (N) {
    case 32: return plan_any_v<T, 32, X>(v, single, batch, members, tiles, s);
    case 64: return plan_any_v<T, 64, X>(v, single, batch, members, tiles, s);
    case 128: return plan_any_v<T, 128, X>(v, single, batch, members, tiles, s);
    case 256: return plan_any_v<T, 256, X>(v, single, batch, members, tiles, s);
    case 512: return plan_any_v<T, 512, X>(v, single, batch, members, tiles, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool X>
int plan_lpc(int N, int v)
{
#define SPSTD_P(n)                                                                                  \
    if (N == n)                                                                                     \
        return v == 1 ? (Plan<T, n, 1, X>::valid ? Plan<T, n, 1, X>::LPC : 0)                       \
             : v == 2 ? (Plan<T, n, 2, X>::valid ? Plan<T, n, 2, X>::LPC : 0)                       \
             : v == 3 ? (Plan<T, n, 3, X>::valid ? Plan<T, n, 3, X>::LPC : 0) : 0;
    SPSTD_P(32) SPSTD_P(64) SPSTD_P(128) SPSTD_P(256) SPSTD_P(512)
#undef SPSTD_P
    return 0;
}

}  // namespace spstd
