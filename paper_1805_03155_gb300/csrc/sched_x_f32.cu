// Schedule variants of the x pass, FP32.
#include "sched_impl.cuh"

namespace spstd {

template <>
cudaError_t xpass_sched<float>(int N, int v, const PassArgs<float> &a, cudaStream_t s)
{
    return plan_any<float, true>(N, v, &a, nullptr, 0, 0, s);
}

template <>
cudaError_t xpass_batch_sched<float>(int N, int v, const PassArgs<float> *args, int members, int tiles, cudaStream_t s)
{
    return plan_any<float, true>(N, v, nullptr, args, members, tiles, s);
}

template <>
int xpass_tiles_sched<float>(int N, int v, int64_t n_rows)
{
    const int lpc = plan_lpc<float, true>(N, v);
    return lpc ? (int)(((n_rows + 1) / 2 + lpc - 1) / lpc) : 0;
}

template <>
bool sched_valid<float>(int axis, int N, int v)
{
    if (!sched_tunable_n(N) || v < 1 || v > 3) return false;
    return axis == 0 ? plan_lpc<float, true>(N, v) > 0 : plan_lpc<float, false>(N, v) > 0;
}

}  // namespace spstd
