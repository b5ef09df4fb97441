// Schedule variants of the strided pass, FP64.
#include "sched_impl.cuh"

namespace spstd {

template <>
cudaError_t spass_sched<double>(int N, int v, const PassArgs<double> &a, cudaStream_t s)
{
    return plan_any<double, false>(N, v, &a, nullptr, 0, 0, s);
}

template <>
cudaError_t spass_batch_sched<double>(int N, int v, const PassArgs<double> *args, int members, int tiles, cudaStream_t s)
{
    return plan_any<double, false>(N, v, nullptr, args, members, tiles, s);
}

template <>
int spass_tiles_sched<double>(int N, int v, int nx, int64_t n_outer)
{
    const int lpc = plan_lpc<double, false>(N, v);
    return lpc ? (int)(((nx + 2 * lpc - 1) / (2 * lpc)) * n_outer) : 0;
}

}  // namespace spstd
