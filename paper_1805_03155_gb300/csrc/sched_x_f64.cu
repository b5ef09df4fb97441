// Schedule variants of the x pass, FP64.
#include "sched_impl.cuh"

namespace spstd {

template <>
cudaError_t xpass_sched<double>(int N, int v, const PassArgs<double> &a, cudaStream_t s)
{
    return plan_any<double, true>(N, v, &a, nullptr, 0, 0, s);
}

template <>
cudaError_t xpass_batch_sched<double>(int N, int v, const PassArgs<double> *args, int members, int tiles, cudaStream_t s)
{
    return plan_any<double, true>(N, v, nullptr, args, members, tiles, s);
}

template <>
int xpass_tiles_sched<double>(int N, int v, int64_t n_rows)
{
    const int lpc = plan_lpc<double, true>(N, v);
    return lpc ? (int)(((n_rows + 1) / 2 + lpc - 1) / lpc) : 0;
}

template <>
bool sched_valid<double>(int axis, int N, int v)
{
    if (!sched_tunable_n(N) || v < 1 || v > 3) return false;
    return axis == 0 ? plan_lpc<double, true>(N, v) > 0 : plan_lpc<double, false>(N, v) > 0;
}

}  // namespace spstd
