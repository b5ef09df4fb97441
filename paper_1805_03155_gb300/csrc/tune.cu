// tune.cu -- the per-context autotuner and the schedule calls of the C ABI
// (include/spstd.h): each axis's candidate pass plans timed on the
// context's own grid, and the x-y fusion switches.
#include "driver.cuh"

using namespace spstd_host;

// ---- autotuner ---------------------------------------------------------------
namespace {

// Schedules an axis of this context can run (sched.h): 0 always; 1..3 for
// plain FFT passes of tunable length; 4 and 5 where 0 is the pipelined TMA
// pass; 6 for x axes that take per-warp tiles; on a dense axis whose 0 is the
// tensor-core pass, 4 (the CUDA-core dense pass).
int schedule_candidates(const spstd_ctx *ctx, int ax, int *list)
{
    int n = 0;
    list[n++] = 0;
    if (ax >= 0 && ax < ctx->cfg.dims && ctx->dense[ax] && dense_tc_axis(ctx->cfg, ax)) list[n++] = 4;
    if (ax < 0 || ax >= ctx->cfg.dims || ctx->dense[ax] || (ax == 0 && ctx->long_x)) return n;
    const int N = (int)ctx->cfg.n[ax];
    for (int v = 1; v <= 3; ++v) {
        const bool ok = ctx->cfg.precision == 32 ? sched_valid<float>(ax, N, v) : sched_valid<double>(ax, N, v);
        if (ok) list[n++] = v;
    }
    if (ctx->tma[ax]) list[n++] = 4;
    if (ctx->tma[ax] && ctx->tma_st[ax]) list[n++] = 5;
    if (ax == 0 && ctx->xw_ok) list[n++] = 6;
    return n;
}

// Times every candidate schedule of every axis on this context's own grid: the
// pass applies H to psi_I into the scratch field (the state is not touched),
// once to warm up, then reps times between two events.  Keeps the fastest.
template <typename T>
spstd_status tune_impl(spstd_ctx *ctx, int reps, double *ms)
{
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPSTD_CU(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, SPSTD_ECUDA, "cudaEventCreate");
    }
    spstd_status st = SPSTD_OK;
    const int tH = 2 * ctx->m;
    for (int ax = 0; ax < ctx->cfg.dims && st == SPSTD_OK; ++ax) {
        int list[kSchedules];
        const int nc = schedule_candidates(ctx, ax, list);
        int best = ctx->sched[ax];
        double best_ms = 0.0;
        for (int i = 0; i < nc && st == SPSTD_OK; ++i) {
            ctx->sched[ax] = list[i];
            st = prepare_kernels<T>(ctx);
            if (st != SPSTD_OK) break;
            cudaError_t e = enqueue_apply<T>(ctx, 1, 2, tH, 1.0, 0, s, nullptr, ax);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_apply<T>(ctx, 1, 2, tH, 1.0, 0, s, nullptr, ax);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                st = cuda_fail(ctx, e, "autotune");
                break;
            }
            const double per = (double)t / reps;
            if (ms) ms[ax * kSchedules + list[i]] = per;
            if (i == 0 || per < best_ms) {
                best_ms = per;
                best = list[i];
            }
        }
        ctx->sched[ax] = best;
    }
    // x and y as separate passes, the stored-tile fused x-y pass or the fused
    // reduce-add x-y pass: time a whole H-apply each way and keep the fastest
    const bool old_ok = xy_fusable(ctx->cfg) && ctx->tma_st[0] && ctx->tma_st[1];
    if (st == SPSTD_OK && (old_ok || ctx->fxy_ok) && ctx->sched[0] == 0 && ctx->sched[1] == 0) {
        double best_t = 0.0;
        int best = 0;
        for (int f = 0; f < 3 && st == SPSTD_OK; ++f) {
            if ((f == 1 && !old_ok) || (f == 2 && !ctx->fxy_ok)) continue;
            ctx->fuse_xy = f == 1;
            ctx->fxy_on = f == 2;
            st = prepare_kernels<T>(ctx);
            if (st != SPSTD_OK) break;
            cudaError_t e = enqueue_apply<T>(ctx, 1, 2, tH, 1.0, 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_apply<T>(ctx, 1, 2, tH, 1.0, 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) st = cuda_fail(ctx, e, "autotune");
            if (f == 0 || t < best_t) {
                best_t = t;
                best = f;
            }
        }
        ctx->fuse_xy = best == 1;
        ctx->fxy_on = best == 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graph(ctx);
    if (st == SPSTD_OK) st = check_device_status(ctx);
    return st;
}

}  // namespace

extern "C" {

spstd_status spstd_schedule_candidates(const spstd_ctx *ctx, int axis, int *list, int *count)
{
    if (!ctx || !list || !count || axis < 0 || axis >= ctx->cfg.dims) return SPSTD_EINVAL;
    *count = schedule_candidates(ctx, axis, list);
    return SPSTD_OK;
}

spstd_status spstd_get_schedule(const spstd_ctx *ctx, int axis, int *schedule)
{
    if (!ctx || !schedule || axis < 0 || axis >= ctx->cfg.dims) return SPSTD_EINVAL;
    *schedule = ctx->sched[axis];
    return SPSTD_OK;
}

spstd_status spstd_set_schedule(spstd_ctx *ctx, int axis, int schedule)
{
    if (!ctx || axis < 0 || axis >= ctx->cfg.dims) return SPSTD_EINVAL;
    int list[kSchedules];
    const int nc = schedule_candidates(ctx, axis, list);
    bool ok = false;
    for (int i = 0; i < nc; ++i) ok |= list[i] == schedule;
    if (!ok) return fail(ctx, SPSTD_EINVAL, "schedule not available on this axis");
    if (ctx->sched[axis] != schedule) {
        ctx->sched[axis] = schedule;
        drop_graph(ctx);
    }
    return SPSTD_OK;
}

spstd_status spstd_set_xy_fusion(spstd_ctx *ctx, int on)
{
    if (!ctx) return SPSTD_EINVAL;
    const bool can = xy_fusable(ctx->cfg) && ctx->tma_st[0] && ctx->tma_st[1];
    if (on && !can) return fail(ctx, SPSTD_EUNSUPPORTED, "x-y fusion needs a 3D FP32 grid with nx = ny in {64, 128, 256}");
    if (ctx->fuse_xy != (on != 0)) {
        ctx->fuse_xy = on != 0;
        drop_graph(ctx);
    }
    return SPSTD_OK;
}

spstd_status spstd_inject_wait_timeout(spstd_ctx *ctx)
{
    if (!ctx) return SPSTD_EINVAL;
    if (!fused_active(ctx) && ctx->tma[0] && (ctx->sched[0] == 0 || (ctx->sched[0] == 6 && ctx->xw_ok))) {
        // the next default x pass leaves its first tile unloaded: the word after
        // the status word is its injection flag
        const int one = 1;
        SPSTD_CU(ctx, cudaMemcpyAsync((int *)ctx->ptr(ctx->L.status) + 1, &one, sizeof(one), cudaMemcpyHostToDevice,
                                      ctx->stream));
        SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
        return SPSTD_OK;
    }
    if (!fused_active(ctx)) return fail(ctx, SPSTD_EUNSUPPORTED, "no pipelined pass to stall");
    // the next fused pass starts its work list at item 1: the first y tile of
    // plane 0 is never claimed, so that plane's x tiles wait in vain
    const unsigned first = 1u;
    SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.xy), &first, sizeof(first), cudaMemcpyHostToDevice, ctx->stream));
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return SPSTD_OK;
}

spstd_status spstd_get_xy_fusion(const spstd_ctx *ctx, int *on)
{
    if (!ctx || !on) return SPSTD_EINVAL;
    *on = fused_active(ctx) ? 1 : 0;
    return SPSTD_OK;
}

spstd_status spstd_tune(spstd_ctx *ctx, int reps, double *ms)
{
    if (!ctx || reps < 1) return SPSTD_EINVAL;
    NvtxRange r("spstd_tune");
    if (ms)
        for (int i = 0; i < 3 * kSchedules; ++i) ms[i] = -1.0;
    return ctx->cfg.precision == 32 ? tune_impl<float>(ctx, reps, ms) : tune_impl<double>(ctx, reps, ms);
}

}  // extern "C"
