// batch.cu -- the batch calls of the C ABI (include/spstd.h): many
// independent solves advanced together, their HBM-cap admission, the batched
// pass launches captured in CUDA graphs, and the batch autotuner.
#include "driver.cuh"

using namespace spstd_host;

// =============================================================================
// Batches: many independent solves advanced together.
//
// Members are grouped by shape: 1D members of one length and precision run
// every step of a call in one resident block each (one launch per group, on a
// side stream); 2D/3D members sharing dims, sizes, precision and integrator
// run each pass of each half-stage as one batched launch over all members'
// tiles (descriptors per member: its own fields, V, dt-scaled multipliers,
// probes).  Chunks of steps are replayed from one captured CUDA graph, whose
// groups follow one another: each batched pass fills the GPU, and groups on
// parallel branches (the fork option of enqueue_nd_steps) measured 4 % slower
// on the 512-solve mix, their persistent blocks competing for the SMs.
// =============================================================================
namespace {

constexpr int kBatchGraphSteps = 10;
constexpr int kBatchStreams = 4;
constexpr size_t kBatchBytesPerMember = 16384;

struct BatchGroup1D {
    int precision;
    int64_t N;
    std::vector<int> slots;
    size_t args_off;
};

struct BatchGroupND {
    int precision, dims, m;
    int64_t n[3];
    double c[SPSTD_MAX_STAGES], d[SPSTD_MAX_STAGES];
    std::vector<int> slots;
    int nh;
    int tiles[3];
    int sched[3];      // pass schedule per axis (0..4; 0 is the TMA pass where tma[ax])
    bool tma[3];       // axis can run the batched reduce-add TMA pass
    bool fxy;          // x and y run as the batched fused x-y pass (while both are on schedule 0)
    bool vsep;         // every member has separable-potential tables: the x pass takes the table form
    bool xw;           // every member has per-warp x maps: the x axis may run schedule 6
    size_t args_off;   // PassArgs<T> [nh * dims][M]
    size_t probe_off;  // ProbeMember<T> [M]
    size_t tma_off;    // TmaMember [M] (when any tma[ax])
    const void *tw[3]; // twiddle table per axis (identical in every member; the first member's)
};

}  // namespace

// A schedule the batch autotuner chose for one member shape.
struct TunedShape {
    int precision, dims;
    int64_t n[3];
    int sched[3];
};

struct spstd_batch {
    int device = 0;
    int max_members = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t branch[kBatchStreams] = {nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_branch[kBatchStreams] = {nullptr};
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t hbm_cap = 0;     // cap on the members' workspaces (0: none)
    size_t in_use = 0;      // sum of the members' workspace bytes
    std::vector<spstd_ctx *> slots;
    bool dirty = true;
    std::vector<BatchGroup1D> g1;
    std::vector<BatchGroupND> gn;
    std::vector<TunedShape> tuned;
    size_t img_bytes = 0;  // descriptor image size (the tuner's scratch descriptors follow it)
    cudaGraphExec_t gexec = nullptr;
    std::string err;
};

namespace {

spstd_status bfail(spstd_batch *b, spstd_status s, const std::string &msg)
{
    if (b) b->err = msg;
    return s;
}
#define SPSTD_BCU(b, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return bfail(b, SPSTD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool same_integrator(const spstd_ctx *a, int m, const double *c, const double *d)
{
    if (a->m != m) return false;
    for (int l = 0; l < m; ++l)
        if (a->c[l] != c[l] || a->d[l] != d[l]) return false;
    return true;
}

template <typename T>
PassArgs<T> member_pass_args(spstd_ctx *ctx, const HalfStage &h, int ax)
{
    const spstd_config &cfg = ctx->cfg;
    const int64_t n0 = cfg.n[0], n1 = cfg.n[1], n2 = cfg.n[2];
    const int64_t *off = ctx->tab_off;
    PassArgs<T> a{};
    a.src = field_ptr<T>(ctx, 1 - h.dst);
    a.dst = field_ptr<T>(ctx, h.dst);
    a.tw = (const cpx<T> *)ctx->ptr(ctx->L.tw[ax]);
    a.mult = (const T *)ctx->ptr(ctx->L.mult) + (size_t)h.table * ctx->sum_n + off[ax];
    if (ax == 0) {
        a.V = (const T *)ctx->ptr(ctx->L.V);
        a.bV = (T)h.bV;
        a.use_V = 1;
        a.n_rows = n1 * n2;
        if constexpr (sizeof(T) == 4) {
            if (ctx->vsep) {
                a.vx = (const T *)ctx->ptr(ctx->L.vsep_x);
                a.vyz = (const T *)ctx->ptr(ctx->L.vsep_yz);
            }
        }
    } else {
        a.stride = ax == 1 ? n0 : n0 * n1;
        a.outer_stride = ax == 1 ? n0 * n1 : n0;
        a.n_outer = ax == 1 ? n2 : n1;
        a.nx = (int)n0;
    }
    return a;
}

template <typename T>
ResidentArgs<T> member_resident_args(spstd_ctx *ctx)
{
    ResidentArgs<T> r{};
    r.psiR = field_ptr<T>(ctx, 0);
    r.psiI = field_ptr<T>(ctx, 1);
    r.V = (const T *)ctx->ptr(ctx->L.V);
    r.tw = (const cpx<T> *)ctx->ptr(ctx->L.tw[0]);
    r.mult = (const T *)ctx->ptr(ctx->L.mult);
    r.nh = (int)ctx->hs.size();
    for (int h = 0; h < r.nh; ++h) {
        r.bV[h] = (T)ctx->hs[h].bV;
        r.hfield[h] = ctx->hs[h].dst;
        r.htable[h] = ctx->hs[h].table;
    }
    ProbeArgs p = probe_args<float>(ctx);
    r.n_probe = p.n_probe;
    for (int q = 0; q < p.n_probe; ++q) r.probe_idx[q] = p.idx[q];
    r.ring = p.ring;
    r.cap = p.cap;
    r.counter = p.counter;
    return r;
}

// Appends bytes to the descriptor image, 256-byte aligned; returns the offset.
size_t put(std::vector<unsigned char> &img, const void *src, size_t bytes)
{
    size_t off = (img.size() + 255) & ~size_t(255);
    img.resize(off + bytes);
    std::memcpy(img.data() + off, src, bytes);
    return off;
}

// Whether schedule v of axis ax runs the batched TMA pass.
// Schedules of a batched pass (sched.h): 0 the reduce-add TMA pass (block
// tiles) where g.tma[ax], 6 its per-warp x tiles where g.xw, 1..4 plain plans.
bool group_uses_tma(const BatchGroupND &g, int ax, int v)
{
    return (v == 0 && g.tma[ax]) || (v == 6 && ax == 0 && g.xw);
}

// Blocks per member of a batched pass of axis ax under schedule v (4: the
// plain default where 0 is the TMA pass).
template <typename T>
int group_tiles(const BatchGroupND &g, int ax, int v)
{
    if (v == 6 && group_uses_tma(g, ax, v)) {
        const int R = xwarp_rows((int)g.n[0]);
        return (int)((g.n[1] * g.n[2] + R - 1) / R);
    }
    if (group_uses_tma(g, ax, v)) return tmared_tiles(ax, g.n, nullptr);
    if (v == 4) v = 0;
    if (ax == 0)
        return v ? xpass_tiles_sched<T>((int)g.n[0], v, g.n[1] * g.n[2])
                 : Launch<T>::xpass_tiles((int)g.n[0], g.n[1] * g.n[2]);
    const int64_t outer = ax == 1 ? g.n[2] : g.n[1];
    return v ? spass_tiles_sched<T>((int)g.n[ax], v, (int)g.n[0], outer)
             : Launch<T>::spass_tiles((int)g.n[ax], (int)g.n[0], outer);
}

// One batched pass of axis ax under schedule v (no work: raises the smem
// limit).  The TMA pass reads field src (or 1 - dst when src < 0) of each
// member through mem and accumulates into field dst.
template <typename T>
cudaError_t group_pass(const BatchGroupND &g, int ax, int v, const PassArgs<T> *a, int M, int tiles, cudaStream_t s,
                       const TmaMember *mem = nullptr, int src = -1, int dst = 0)
{
    const int N = (int)g.n[ax];
    if constexpr (sizeof(T) == 4) {
        if (group_uses_tma(g, ax, v)) {
            if (!a) return v == 6 ? prepare_pass_xwarp_batch(N) : prepare_pass_tmared_batch(ax, N, g.n[0], red_planes(g.n, ax));
            TmaBatchArgs ta{};
            ta.mem = mem;
            ta.pa = a;
            ta.tw = (const float2 *)g.tw[ax];
            ta.src = src;
            ta.dst = dst;
            ta.members = M;
            ta.tiles = tiles;
            tmared_tiles(ax, g.n, &ta.n_xt);
            ta.nx = (int)g.n[0];
            ta.planes = red_planes(g.n, ax);
            ta.vsep = ax == 0 && g.vsep;
            ta.axis = ax;
            return v == 6 ? launch_pass_xwarp_batch(N, ta, s) : launch_pass_tmared_batch(ax, N, ta, s);
        }
    }
    if (v == 4) v = 0;
    if (ax == 0) return v ? xpass_batch_sched<T>(N, v, a, M, tiles, s) : Launch<T>::xpass_batch(N, a, M, tiles, s);
    return v ? spass_batch_sched<T>(N, v, a, M, tiles, s) : Launch<T>::spass_batch(N, a, M, tiles, s);
}

template <typename T>
void build_nd_descriptors(spstd_batch *b, BatchGroupND &g, std::vector<unsigned char> &img)
{
    const int M = (int)g.slots.size();
    std::vector<PassArgs<T>> args((size_t)g.nh * g.dims * M);
    std::vector<ProbeMember<T>> pm(M);
    for (int i = 0; i < M; ++i) {
        spstd_ctx *ctx = b->slots[g.slots[i]];
        for (int h = 0; h < g.nh; ++h)
            for (int ax = 0; ax < g.dims; ++ax)
                args[((size_t)h * g.dims + ax) * M + i] = member_pass_args<T>(ctx, ctx->hs[h], ax);
        pm[i].psiR = field_ptr<T>(ctx, 0);
        pm[i].psiI = field_ptr<T>(ctx, 1);
        pm[i].p = probe_args<T>(ctx);
    }
    g.args_off = put(img, args.data(), sizeof(PassArgs<T>) * args.size());
    g.probe_off = put(img, pm.data(), sizeof(ProbeMember<T>) * pm.size());
    // batched TMA passes: FP32 axes where every member has its tensor maps and
    // 16-byte aligned multiplier rows (the stage's bulk copy needs both)
    bool any = false;
    for (int ax = 0; ax < 3; ++ax) {
        g.tw[ax] = b->slots[g.slots[0]]->ptr(b->slots[g.slots[0]]->L.tw[ax]);
        bool ok = sizeof(T) == 4 && ax < g.dims;
        for (int i = 0; i < M && ok; ++i) {
            spstd_ctx *ctx = b->slots[g.slots[i]];
            ok = ctx->tma[ax];
            for (int h = 0; h < g.nh && ok; ++h)
                ok = ((uintptr_t)args[((size_t)h * g.dims + ax) * M + i].mult & 15) == 0;
        }
        g.tma[ax] = ok;
        any |= ok;
    }
    g.tma_off = 0;
    g.vsep = g.tma[0];
    for (int i = 0; i < M && g.vsep; ++i) g.vsep = b->slots[g.slots[i]]->vsep;
    g.xw = g.tma[0];
    for (int i = 0; i < M && g.xw; ++i) g.xw = b->slots[g.slots[i]]->xw_ok;
    g.fxy = any && g.tma[0] && g.tma[1];
    for (int i = 0; i < M && g.fxy; ++i) g.fxy = b->slots[g.slots[i]]->fxy_ok && b->slots[g.slots[i]]->fxy_on;
    if (any) {
        std::vector<TmaMember> tm(M);
        for (int i = 0; i < M; ++i) {
            spstd_ctx *ctx = b->slots[g.slots[i]];
            TmaMember &t = tm[i];
            std::memset(&t, 0, sizeof(t));
            for (int f = 0; f < 4; ++f) {
                if (g.tma[0]) t.x[f] = ctx->xrmap[f];
                if (g.xw) t.xw[f] = ctx->xwmap[f];
            }
            for (int f = 0; f < 3; ++f) {
                if (g.tma[1]) t.y[f] = ctx->srmap[f][0];
                if (g.tma[2]) t.z[f] = ctx->srmap[f][1];
            }
            if (g.fxy)
                for (int f = 0; f < 4; ++f) t.f[f] = ctx->fxmap[f];
            t.status = (int *)ctx->ptr(ctx->L.status);
        }
        g.tma_off = put(img, tm.data(), sizeof(TmaMember) * tm.size());
    }
    // a tuned per-warp x schedule needs every member's per-warp maps
    if (g.sched[0] == 6 && !g.xw) g.sched[0] = 0;
    for (int ax = 0; ax < g.dims; ++ax) g.tiles[ax] = group_tiles<T>(g, ax, g.sched[ax]);
}

template <typename T>
void build_1d_descriptors(spstd_batch *b, BatchGroup1D &g, std::vector<unsigned char> &img)
{
    std::vector<ResidentArgs<T>> args(g.slots.size());
    for (size_t i = 0; i < g.slots.size(); ++i) args[i] = member_resident_args<T>(b->slots[g.slots[i]]);
    g.args_off = put(img, args.data(), sizeof(ResidentArgs<T>) * args.size());
}

spstd_status batch_build(spstd_batch *b)
{
    b->g1.clear();
    b->gn.clear();
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        spstd_ctx *ctx = b->slots[s];
        if (!ctx) continue;
        const spstd_config &cfg = ctx->cfg;
        if (cfg.dims == 1) {
            BatchGroup1D *g = nullptr;
            for (auto &x : b->g1)
                if (x.precision == cfg.precision && x.N == cfg.n[0]) g = &x;
            if (!g) {
                b->g1.push_back(BatchGroup1D{cfg.precision, cfg.n[0], {}, 0});
                g = &b->g1.back();
            }
            g->slots.push_back(s);
        } else {
            BatchGroupND *g = nullptr;
            for (auto &x : b->gn)
                if (x.precision == cfg.precision && x.dims == cfg.dims && x.n[0] == cfg.n[0] && x.n[1] == cfg.n[1] &&
                    x.n[2] == cfg.n[2] && x.nh == (int)ctx->hs.size() && same_integrator(ctx, x.m, x.c, x.d))
                    g = &x;
            if (!g) {
                BatchGroupND ng{};
                ng.precision = cfg.precision;
                ng.dims = cfg.dims;
                ng.m = ctx->m;
                for (int a = 0; a < 3; ++a) ng.n[a] = cfg.n[a];
                for (int l = 0; l < ctx->m; ++l) {
                    ng.c[l] = ctx->c[l];
                    ng.d[l] = ctx->d[l];
                }
                ng.nh = (int)ctx->hs.size();
                for (const TunedShape &t : b->tuned)
                    if (t.precision == ng.precision && t.dims == ng.dims && t.n[0] == ng.n[0] && t.n[1] == ng.n[1] &&
                        t.n[2] == ng.n[2])
                        for (int a = 0; a < 3; ++a) ng.sched[a] = t.sched[a];
                b->gn.push_back(ng);
                g = &b->gn.back();
            }
            g->slots.push_back(s);
        }
    }
    std::vector<unsigned char> img;
    for (auto &g : b->g1) {
        if (g.precision == 32) build_1d_descriptors<float>(b, g, img);
        else build_1d_descriptors<double>(b, g, img);
    }
    for (auto &g : b->gn) {
        if (g.precision == 32) build_nd_descriptors<float>(b, g, img);
        else build_nd_descriptors<double>(b, g, img);
    }
    if (img.size() > b->ws_bytes) return bfail(b, SPSTD_ENOMEM, "batch workspace too small for the descriptors");
    b->img_bytes = img.size();
    if (!img.empty()) {
        SPSTD_BCU(b, cudaMemcpyAsync(b->ws, img.data(), img.size(), cudaMemcpyHostToDevice, b->stream));
        SPSTD_BCU(b, cudaStreamSynchronize(b->stream));
    }
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->dirty = false;
    return SPSTD_OK;
}

template <typename T>
cudaError_t enqueue_group_step(spstd_batch *b, const BatchGroupND &g, cudaStream_t s)
{
    const int M = (int)g.slots.size();
    const PassArgs<T> *args = (const PassArgs<T> *)(b->ws + g.args_off);
    const TmaMember *mem = (const TmaMember *)(b->ws + g.tma_off);
    const spstd_ctx *first = b->slots[g.slots[0]];
    const bool fxy = sizeof(T) == 4 && g.fxy && g.sched[0] == 0 && g.sched[1] == 0;
    for (int h = 0; h < g.nh; ++h) {
        int ax0 = 0;
        if constexpr (sizeof(T) == 4) {
            if (fxy) {
                TmaBatchArgs fa{};
                fa.mem = mem;
                fa.pa = (const PassArgs<float> *)(args + ((size_t)h * g.dims + 0) * M);
                fa.pa_y = (const PassArgs<float> *)(args + ((size_t)h * g.dims + 1) * M);
                fa.tw = (const float2 *)g.tw[0];
                fa.src = -1;
                fa.dst = first->hs[h].dst;
                fa.members = M;
                fa.tiles = fxy_units(g.n);
                cudaError_t e = launch_pass_fxy_batch((int)g.n[0], fa, s);
                if (e != cudaSuccess) return e;
                ax0 = 2;
            }
        }
        for (int ax = ax0; ax < g.dims; ++ax) {
            const PassArgs<T> *a = args + ((size_t)h * g.dims + ax) * M;
            cudaError_t e = group_pass<T>(g, ax, g.sched[ax], a, M, g.tiles[ax], s, mem, -1, first->hs[h].dst);
            if (e != cudaSuccess) return e;
        }
    }
    return Launch<T>::probe_batch((const ProbeMember<T> *)(b->ws + g.probe_off), M, s);
}

cudaError_t enqueue_nd_steps(spstd_batch *b, int64_t nsteps, cudaStream_t s, bool fork)
{
    for (int64_t i = 0; i < nsteps; ++i) {
        if (fork && b->gn.size() > 1) {
            cudaError_t e = cudaEventRecord(b->ev_fork, s);
            if (e != cudaSuccess) return e;
            for (size_t g = 0; g < b->gn.size(); ++g) {
                cudaStream_t bs = b->branch[g % kBatchStreams];
                if (g < kBatchStreams) {
                    e = cudaStreamWaitEvent(bs, b->ev_fork, 0);
                    if (e != cudaSuccess) return e;
                }
                e = b->gn[g].precision == 32 ? enqueue_group_step<float>(b, b->gn[g], bs)
                                             : enqueue_group_step<double>(b, b->gn[g], bs);
                if (e != cudaSuccess) return e;
            }
            for (int k = 0; k < kBatchStreams && k < (int)b->gn.size(); ++k) {
                e = cudaEventRecord(b->ev_branch[k], b->branch[k]);
                if (e != cudaSuccess) return e;
                e = cudaStreamWaitEvent(s, b->ev_branch[k], 0);
                if (e != cudaSuccess) return e;
            }
        } else {
            for (const auto &g : b->gn) {
                cudaError_t e = g.precision == 32 ? enqueue_group_step<float>(b, g, s)
                                                  : enqueue_group_step<double>(b, g, s);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

// Raises the shared-memory limits of every batched kernel used (outside any capture).
cudaError_t batch_prepare(spstd_batch *b)
{
    for (const auto &g : b->gn) {
        for (int ax = 0; ax < g.dims; ++ax) {
            cudaError_t e = g.precision == 32 ? group_pass<float>(g, ax, g.sched[ax], nullptr, 0, 0, nullptr)
                                              : group_pass<double>(g, ax, g.sched[ax], nullptr, 0, 0, nullptr);
            if (e != cudaSuccess) return e;
        }
        if (g.fxy) {
            cudaError_t e = prepare_pass_fxy((int)g.n[0], true);
            if (e != cudaSuccess) return e;
        }
    }
    for (const auto &g : b->g1) {
        cudaError_t e = g.precision == 32 ? Launch<float>::resident_batch((int)g.N, nullptr, 0, 0, nullptr)
                                          : Launch<double>::resident_batch((int)g.N, nullptr, 0, 0, nullptr);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

namespace spstd_host {
void batch_member_changed(spstd_batch *b)
{
    if (b) b->dirty = true;
}
}  // namespace spstd_host

extern "C" {

spstd_status spstd_batch_workspace_size(int max_members, size_t *bytes)
{
    if (max_members < 1 || !bytes) return SPSTD_EINVAL;
    *bytes = (size_t)max_members * kBatchBytesPerMember + 4096;
    return SPSTD_OK;
}

spstd_status spstd_batch_create(int max_members, size_t hbm_cap_bytes, int device, void *stream, void *d_workspace,
                                size_t workspace_bytes, spstd_batch **out)
{
    if (!out || max_members < 1) return SPSTD_EINVAL;
    *out = nullptr;
    size_t need = 0;
    spstd_batch_workspace_size(max_members, &need);
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return SPSTD_EINVAL;
    if (workspace_bytes < need) return SPSTD_ENOMEM;
    spstd_batch *b = new (std::nothrow) spstd_batch();
    if (!b) return SPSTD_ENOMEM;
    b->device = device;
    b->max_members = max_members;
    b->stream = (cudaStream_t)stream;
    b->ws = (unsigned char *)d_workspace;
    b->ws_bytes = workspace_bytes;
    b->hbm_cap = hbm_cap_bytes;
    b->slots.assign(max_members, nullptr);
    bool ok = cudaSetDevice(device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kBatchStreams; ++k)
        ok = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev_branch[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        spstd_batch_destroy(b);
        return SPSTD_ECUDA;
    }
    *out = b;
    return SPSTD_OK;
}

spstd_status spstd_batch_destroy(spstd_batch *b)
{
    if (!b) return SPSTD_OK;
    if (b->stream || b->side) {
        cudaStreamSynchronize(b->stream);
        if (b->side) cudaStreamSynchronize(b->side);
    }
    for (spstd_ctx *c : b->slots)
        if (c) c->batch = nullptr;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (int k = 0; k < kBatchStreams; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->ev_branch[k]) cudaEventDestroy(b->ev_branch[k]);
    }
    if (b->side) cudaStreamDestroy(b->side);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
    return SPSTD_OK;
}

spstd_status spstd_batch_add(spstd_batch *b, spstd_ctx *ctx, int *slot)
{
    if (!b || !ctx || !slot) return SPSTD_EINVAL;
    if (ctx->batch) return bfail(b, SPSTD_EINVAL, "context is already a batch member");
    if (ctx->cfg.device != b->device) return bfail(b, SPSTD_EINVAL, "context lives on another device");
    for (int a = 0; a < ctx->cfg.dims; ++a)
        if (ctx->dense[a])
            return bfail(b, SPSTD_EUNSUPPORTED, "batches take FFT axes only (periodic; powers of two, or 3 * 2^k "
                                                "for 24..384 in 2D/3D)");
    if (ctx->rk4) return bfail(b, SPSTD_EUNSUPPORTED, "batches take the partitioned symplectic schemes only");
    if (ctx->long_x) return bfail(b, SPSTD_EUNSUPPORTED, "batches take lines of at most 8192 (1D) / 1024 points");
    // admission by device footprint: the member's workspace must fit under the cap
    const size_t need = ctx->L.total;
    if (b->hbm_cap && need > b->hbm_cap) return bfail(b, SPSTD_EINVAL, "member workspace exceeds the batch's HBM cap");
    if (b->hbm_cap && b->in_use + need > b->hbm_cap) return bfail(b, SPSTD_ENOTREADY, "HBM cap reached");
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        if (!b->slots[s]) {
            // the member's own pending work comes first
            SPSTD_BCU(b, cudaStreamSynchronize(ctx->stream));
            b->slots[s] = ctx;
            ctx->batch = b;
            b->in_use += need;
            b->dirty = true;
            *slot = s;
            return SPSTD_OK;
        }
    }
    return bfail(b, SPSTD_ENOTREADY, "batch is full");
}

spstd_status spstd_batch_remove(spstd_batch *b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot]) return SPSTD_EINVAL;
    SPSTD_BCU(b, cudaStreamSynchronize(b->stream));
    b->in_use -= b->slots[slot]->L.total;
    b->slots[slot]->batch = nullptr;
    b->slots[slot] = nullptr;
    b->dirty = true;
    return SPSTD_OK;
}

spstd_status spstd_batch_footprint(const spstd_batch *b, size_t *in_use, size_t *cap)
{
    if (!b || !in_use || !cap) return SPSTD_EINVAL;
    *in_use = b->in_use;
    *cap = b->hbm_cap;
    return SPSTD_OK;
}

spstd_status spstd_batch_size(const spstd_batch *b, int *members)
{
    if (!b || !members) return SPSTD_EINVAL;
    int n = 0;
    for (auto *c : b->slots) n += c != nullptr;
    *members = n;
    return SPSTD_OK;
}

spstd_status spstd_batch_step(spstd_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0) return SPSTD_EINVAL;
    if (nsteps == 0) return SPSTD_OK;
    NvtxRange r("spstd_batch_step");
    if (b->dirty) {
        spstd_status st = batch_build(b);
        if (st != SPSTD_OK) return st;
        SPSTD_BCU(b, batch_prepare(b));
    }
    // 1D groups: every step of this call in one resident launch each, on the side stream
    if (!b->g1.empty()) {
        SPSTD_BCU(b, cudaEventRecord(b->ev_fork, b->stream));
        SPSTD_BCU(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        for (const auto &g : b->g1) {
            const int M = (int)g.slots.size();
            if (g.precision == 32)
                SPSTD_BCU(b, Launch<float>::resident_batch((int)g.N, (const ResidentArgs<float> *)(b->ws + g.args_off),
                                                           M, nsteps, b->side));
            else
                SPSTD_BCU(b, Launch<double>::resident_batch((int)g.N, (const ResidentArgs<double> *)(b->ws + g.args_off),
                                                            M, nsteps, b->side));
        }
    }
    // 2D/3D groups: graph-replayed chunks, then the remainder directly
    int64_t left = nsteps;
    if (!b->gn.empty() && left >= kBatchGraphSteps) {
        if (!b->gexec) {
            cudaGraph_t g = nullptr;
            SPSTD_BCU(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_nd_steps(b, kBatchGraphSteps, b->cap, false);
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bfail(b, SPSTD_ECUDA, std::string("batch graph capture: ") +
                                                 cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return bfail(b, SPSTD_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
            }
        }
        for (int64_t r = 0; r < left / kBatchGraphSteps; ++r) SPSTD_BCU(b, cudaGraphLaunch(b->gexec, b->stream));
        left %= kBatchGraphSteps;
    }
    if (!b->gn.empty() && left > 0) SPSTD_BCU(b, enqueue_nd_steps(b, left, b->stream, false));
    if (!b->g1.empty()) {
        SPSTD_BCU(b, cudaEventRecord(b->ev_join, b->side));
        SPSTD_BCU(b, cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    }
    for (spstd_ctx *c : b->slots)
        if (c) c->steps_taken += nsteps;
    return SPSTD_OK;
}

spstd_status spstd_batch_sync(spstd_batch *b)
{
    if (!b) return SPSTD_EINVAL;
    SPSTD_BCU(b, cudaStreamSynchronize(b->stream));
    return SPSTD_OK;
}

spstd_status spstd_batch_launch_count(const spstd_batch *b, int64_t nsteps, int64_t *launches)
{
    if (!b || !launches || nsteps < 0) return SPSTD_EINVAL;
    int64_t per_step = 0, per_call = 0;
    if (!b->dirty) {
        // built: the groups as they run
        per_call = (int64_t)b->g1.size();
        for (const auto &g : b->gn) {
            const bool fxy = g.precision == 32 && g.fxy && g.sched[0] == 0 && g.sched[1] == 0;
            per_step += (int64_t)g.nh * (g.dims - (fxy ? 1 : 0)) + 1;
        }
    } else {
        // not built yet: group the members the way a build does (one launch per
        // axis; the fused x-y pass is known only after the build)
        std::vector<std::vector<int64_t>> keys;
        for (auto *c : b->slots) {
            if (!c) continue;
            const spstd_config &cfg = c->cfg;
            std::vector<int64_t> k = {cfg.dims, cfg.precision, cfg.n[0], cfg.n[1], cfg.n[2], (int64_t)c->hs.size(),
                                      c->m};
            for (int l = 0; l < c->m; ++l) {
                int64_t bc, bd;
                std::memcpy(&bc, &c->c[l], 8);
                std::memcpy(&bd, &c->d[l], 8);
                k.push_back(bc);
                k.push_back(bd);
            }
            if (cfg.dims == 1) k.resize(3);
            bool found = false;
            for (auto &x : keys) found |= x == k;
            if (found) continue;
            keys.push_back(k);
            if (cfg.dims == 1) ++per_call;
            else per_step += (int64_t)c->hs.size() * cfg.dims + 1;
        }
    }
    *launches = nsteps ? per_call + nsteps * per_step : 0;
    return SPSTD_OK;
}

const char *spstd_batch_last_error(const spstd_batch *b)
{
    return b ? b->err.c_str() : "no batch";
}

}  // extern "C"

// ---- batch autotuner -------------------------------------------------------
namespace {

// Times the batched passes of one member shape under each schedule on the
// members' scratch fields and keeps the fastest per axis; where the group can
// run the fused x-y pass (which schedule 0 on x and y selects), that pass is
// timed against the fastest separate x and y passes.
template <typename T>
spstd_status tune_group(spstd_batch *b, BatchGroupND &g, int reps, cudaEvent_t e0, cudaEvent_t e1)
{
    const int M = (int)g.slots.size();
    const size_t off = (b->img_bytes + 255) & ~size_t(255);
    if (M == 0 || off + 2 * sizeof(PassArgs<T>) * (size_t)M > b->ws_bytes) return SPSTD_OK;  // no room: defaults
    PassArgs<T> *dargs = (PassArgs<T> *)(b->ws + off);
    std::vector<PassArgs<T>> args(M);
    double axis_ms[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < g.dims; ++ax) {
        for (int i = 0; i < M; ++i) {
            spstd_ctx *ctx = b->slots[g.slots[i]];
            args[i] = member_pass_args<T>(ctx, ctx->hs[0], ax);
            args[i].dst = field_ptr<T>(ctx, 2);
        }
        SPSTD_BCU(b, cudaMemcpyAsync(dargs, args.data(), sizeof(PassArgs<T>) * M, cudaMemcpyHostToDevice, b->stream));
        int best = 0;
        double best_ms = 0.0;
        const TmaMember *mem = (const TmaMember *)(b->ws + g.tma_off);
        const int fsrc = 1 - b->slots[g.slots[0]]->hs[0].dst;
        for (int v = 0; v <= 6; ++v) {
            if (v >= 1 && v <= 3 && !sched_valid<T>(ax, (int)g.n[ax], v)) continue;
            if (v == 4 && !g.tma[ax]) continue;
            if (v == 5 || (v == 6 && !group_uses_tma(g, ax, 6))) continue;
            const int tiles = group_tiles<T>(g, ax, v);
            SPSTD_BCU(b, group_pass<T>(g, ax, v, dargs, M, tiles, b->stream, mem, fsrc, 2));
            SPSTD_BCU(b, cudaEventRecord(e0, b->stream));
            for (int r = 0; r < reps; ++r)
                SPSTD_BCU(b, group_pass<T>(g, ax, v, dargs, M, tiles, b->stream, mem, fsrc, 2));
            SPSTD_BCU(b, cudaEventRecord(e1, b->stream));
            SPSTD_BCU(b, cudaEventSynchronize(e1));
            float t = 0.f;
            SPSTD_BCU(b, cudaEventElapsedTime(&t, e0, e1));
            if (v == 0 || t < best_ms) {
                best_ms = t;
                best = v;
            }
        }
        g.sched[ax] = best;
        g.tiles[ax] = group_tiles<T>(g, ax, best);
        axis_ms[ax] = best_ms;
    }
    if constexpr (sizeof(T) == 4) {
        if (g.fxy && (g.sched[0] != 0 || g.sched[1] != 0)) {
            std::vector<PassArgs<T>> xy(2 * (size_t)M);
            for (int i = 0; i < M; ++i) {
                spstd_ctx *ctx = b->slots[g.slots[i]];
                for (int ax = 0; ax < 2; ++ax) {
                    xy[(size_t)ax * M + i] = member_pass_args<T>(ctx, ctx->hs[0], ax);
                    xy[(size_t)ax * M + i].dst = field_ptr<T>(ctx, 2);
                }
            }
            SPSTD_BCU(b, cudaMemcpyAsync(dargs, xy.data(), sizeof(PassArgs<T>) * 2 * M, cudaMemcpyHostToDevice,
                                         b->stream));
            TmaBatchArgs fa{};
            fa.mem = (const TmaMember *)(b->ws + g.tma_off);
            fa.pa = (const PassArgs<float> *)dargs;
            fa.pa_y = (const PassArgs<float> *)dargs + M;
            fa.tw = (const float2 *)g.tw[0];
            fa.src = 1 - b->slots[g.slots[0]]->hs[0].dst;
            fa.dst = 2;
            fa.members = M;
            fa.tiles = fxy_units(g.n);
            SPSTD_BCU(b, launch_pass_fxy_batch((int)g.n[0], fa, b->stream));
            SPSTD_BCU(b, cudaEventRecord(e0, b->stream));
            for (int r = 0; r < reps; ++r) SPSTD_BCU(b, launch_pass_fxy_batch((int)g.n[0], fa, b->stream));
            SPSTD_BCU(b, cudaEventRecord(e1, b->stream));
            SPSTD_BCU(b, cudaEventSynchronize(e1));
            float t = 0.f;
            SPSTD_BCU(b, cudaEventElapsedTime(&t, e0, e1));
            if (t < axis_ms[0] + axis_ms[1]) {
                g.sched[0] = g.sched[1] = 0;
                for (int ax = 0; ax < 2; ++ax) g.tiles[ax] = group_tiles<T>(g, ax, 0);
            }
        }
    }
    TunedShape ts{g.precision, g.dims, {g.n[0], g.n[1], g.n[2]}, {g.sched[0], g.sched[1], g.sched[2]}};
    bool found = false;
    for (TunedShape &t : b->tuned)
        if (t.precision == ts.precision && t.dims == ts.dims && t.n[0] == ts.n[0] && t.n[1] == ts.n[1] &&
            t.n[2] == ts.n[2]) {
            t = ts;
            found = true;
        }
    if (!found) b->tuned.push_back(ts);
    return SPSTD_OK;
}

}  // namespace

extern "C" {

spstd_status spstd_batch_tune(spstd_batch *b, int reps)
{
    if (!b || reps < 1) return SPSTD_EINVAL;
    NvtxRange r("spstd_batch_tune");
    if (b->dirty) {
        spstd_status st = batch_build(b);
        if (st != SPSTD_OK) return st;
    }
    SPSTD_BCU(b, cudaStreamSynchronize(b->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPSTD_BCU(b, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(b, SPSTD_ECUDA, "cudaEventCreate");
    }
    spstd_status st = SPSTD_OK;
    for (auto &g : b->gn) {
        st = g.precision == 32 ? tune_group<float>(b, g, reps, e0, e1) : tune_group<double>(b, g, reps, e0, e1);
        if (st != SPSTD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return st;
}

spstd_status spstd_batch_set_schedule(spstd_batch *b, int precision, int dims, const int64_t *n, const int *schedule)
{
    if (!b || !n || !schedule || (precision != 32 && precision != 64) || dims < 2 || dims > 3) return SPSTD_EINVAL;
    TunedShape ts{precision, dims, {n[0], dims > 1 ? n[1] : 1, dims > 2 ? n[2] : 1}, {0, 0, 0}};
    for (int a = 0; a < dims; ++a) {
        const int v = schedule[a];
        const bool ok = v == 0 || v == 4 || (v == 6 && a == 0 && precision == 32 && xwarp_eligible(n[0])) ||
                        (v >= 1 && v <= 3 &&
                         (precision == 32 ? sched_valid<float>(a, (int)n[a], v) : sched_valid<double>(a, (int)n[a], v)));
        if (!ok) return bfail(b, SPSTD_EINVAL, "schedule not available for this shape and axis");
        ts.sched[a] = v;
    }
    bool found = false;
    for (TunedShape &t : b->tuned)
        if (t.precision == ts.precision && t.dims == ts.dims && t.n[0] == ts.n[0] && t.n[1] == ts.n[1] &&
            t.n[2] == ts.n[2]) {
            t = ts;
            found = true;
        }
    if (!found) b->tuned.push_back(ts);
    b->dirty = true;  // groups pick the schedule up when the batch is rebuilt
    return SPSTD_OK;
}

spstd_status spstd_batch_get_schedule(const spstd_batch *b, int precision, int dims, const int64_t *n, int *schedule)
{
    if (!b || !n || !schedule) return SPSTD_EINVAL;
    for (int a = 0; a < 3; ++a) schedule[a] = 0;
    for (const TunedShape &t : b->tuned)
        if (t.precision == precision && t.dims == dims && t.n[0] == n[0] && t.n[1] == n[1] && t.n[2] == n[2])
            for (int a = 0; a < 3; ++a) schedule[a] = t.sched[a];
    return SPSTD_OK;
}

}  // extern "C"
