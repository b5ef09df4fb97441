// api.cu -- the C ABI of include/spstd.h for single contexts: configuration
// and workspace, creation, potentials and states, the time-step driver
// (direct launches and captured CUDA graphs), probes, spectra, norm and
// energy, eigenstate accumulation, and the per-launch profile.  The shared
// internals live in driver.cuh; batches in batch.cu; the autotuner in tune.cu.
#include "driver.cuh"

using namespace spstd_host;

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

void spstd_config_init(spstd_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dims = 1;
    cfg->n[0] = 256;
    cfg->n[1] = cfg->n[2] = 1;
    for (int a = 0; a < 3; ++a) {
        cfg->lo[a] = 0.0;
        cfg->hi[a] = 1.0;
    }
    cfg->hbar = 1.0;
    cfg->mass = 1.0;
    cfg->precision = 64;
    cfg->preset = SPSTD_FR4;
    cfg->dt = 0.0;
    cfg->probe_capacity = 1024;
    cfg->norm_drift_limit = 1e-3;
}

const char *spstd_status_string(spstd_status s)
{
    switch (s) {
    case SPSTD_OK: return "ok";
    case SPSTD_EINVAL: return "invalid argument";
    case SPSTD_ENOMEM: return "out of memory / workspace too small";
    case SPSTD_ECUDA: return "CUDA error";
    case SPSTD_EUNSTABLE: return "time step above the stability limit";
    case SPSTD_EDIVERGED: return "solution diverged (NaN/Inf)";
    case SPSTD_ETIMEOUT: return "device wait timed out";
    case SPSTD_ENOTREADY: return "no data yet";
    case SPSTD_EUNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

const char *spstd_last_error(const spstd_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

spstd_status spstd_workspace_size(const spstd_config *cfg, size_t *bytes)
{
    if (!bytes) return SPSTD_EINVAL;
    int m;
    double c[SPSTD_MAX_STAGES], d[SPSTD_MAX_STAGES];
    spstd_status s = validate(cfg, nullptr, &m, c, d);
    if (s != SPSTD_OK) return s;
    if (cfg->dt > 0) {
        const double ss = scheme_s_star(cfg->preset, m, c, d);
        if (cfg->dt > ss / w_max_of(*cfg, 0.0)) return SPSTD_EUNSTABLE;
    }
    *bytes = make_layout(*cfg, m).total;
    return SPSTD_OK;
}

spstd_status spstd_stability_limit(const spstd_config *cfg, double vmax, double *s_star, double *dt_max)
{
    int m;
    double c[SPSTD_MAX_STAGES], d[SPSTD_MAX_STAGES];
    spstd_status s = validate(cfg, nullptr, &m, c, d);
    if (s != SPSTD_OK) return s;
    const double ss = scheme_s_star(cfg->preset, m, c, d);
    if (s_star) *s_star = ss;
    if (dt_max) *dt_max = ss / w_max_of(*cfg, vmax);
    return SPSTD_OK;
}

spstd_status spstd_create(const spstd_config *cfg, void *d_workspace, size_t workspace_bytes, spstd_ctx **out)
{
    if (!out) return SPSTD_EINVAL;
    *out = nullptr;
    spstd_ctx *ctx = new (std::nothrow) spstd_ctx();
    if (!ctx) return SPSTD_ENOMEM;
    std::string why;
    spstd_status st = validate(cfg, &why, &ctx->m, ctx->c, ctx->d);
    if (st != SPSTD_OK) {
        delete ctx;
        return st;
    }
    ctx->cfg = *cfg;
    ctx->L = make_layout(*cfg, ctx->m);
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) {
        delete ctx;
        return SPSTD_EINVAL;
    }
    if (workspace_bytes < ctx->L.total) {
        delete ctx;
        return SPSTD_ENOMEM;
    }
    ctx->ws = (unsigned char *)d_workspace;
    ctx->ntot = cfg->n[0] * cfg->n[1] * cfg->n[2];
    for (int a = 0; a < cfg->dims; ++a) {
        ctx->tab_off[a] = ctx->sum_n;
        ctx->sum_n += table_len(*cfg, a);
    }
    ctx->long_x = axis_is_long(*cfg, 0);
    if (ctx->long_x) long_split(cfg->n[0], &ctx->N1, &ctx->N2);
    ctx->stream = (cudaStream_t)cfg->stream;
    for (int a = 0; a < cfg->dims; ++a) ctx->dense[a] = !axis_is_fft(*cfg, a) && !axis_is_long(*cfg, a);
    ctx->s_star = scheme_s_star(cfg->preset, ctx->m, ctx->c, ctx->d);
    ctx->rk4 = cfg->preset == SPSTD_RK4;
    ctx->dt_auto = !(cfg->dt > 0);
    ctx->dt = -1.0;  // forces the first table upload
    auto bail = [&](spstd_status s) {
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        delete ctx;
        return s;
    };
    if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(SPSTD_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(SPSTD_ECUDA);
    if (cudaMemsetAsync(ctx->ws, 0, ctx->L.total, ctx->stream) != cudaSuccess) return bail(SPSTD_ECUDA);
    for (int g = 0; g < ctx->L.n_guard; ++g)
        if (cudaMemsetAsync(ctx->ws + ctx->L.guard[g], kGuardByte, kGuardBytes, ctx->stream) != cudaSuccess)
            return bail(SPSTD_ECUDA);
    st = set_dt(ctx, 0.0);
    if (st != SPSTD_OK) return bail(st);
    setup_tma(ctx);
    // fused x-y pass: available where xy_fusable holds, off until spstd_set_xy_fusion or
    // spstd_tune selects it (measured slower than the separate passes at 256^3)
    ctx->fuse_xy = false;
    *out = ctx;
    return SPSTD_OK;
}

spstd_status spstd_destroy(spstd_ctx *ctx)
{
    if (!ctx) return SPSTD_OK;
    cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return SPSTD_OK;
}

}  // extern "C"

namespace {
// Tables of a separable potential V(x_i, row r) = vx[i] + vyz[r] (r = the
// flattened (y, z) index), when the FP32 sum of the two reproduces every
// value of V to 4 units in the last place.  The reference point of the split
// is the smallest |V|: for a potential of one sign (a harmonic well) both
// tables then keep that sign and the sum does not cancel.  vyz is padded with
// zeros to `padded` rows.
bool separable_tables(const double *V, int64_t n0, int64_t rows, int64_t padded, std::vector<float> &vx,
                      std::vector<float> &vyz)
{
    int64_t ref = 0;
    for (int64_t p = 1; p < n0 * rows; ++p)
        if (std::fabs(V[p]) < std::fabs(V[ref])) ref = p;
    const int64_t i0 = ref % n0, r0 = ref / n0;
    vx.assign(n0, 0.f);
    vyz.assign(padded, 0.f);
    for (int64_t i = 0; i < n0; ++i) vx[i] = (float)(V[r0 * n0 + i] - V[ref]);
    for (int64_t r = 0; r < rows; ++r) vyz[r] = (float)V[r * n0 + i0];
    for (int64_t r = 0; r < rows; ++r) {
        const float b = vyz[r];
        const double *row = V + r * n0;
        for (int64_t i = 0; i < n0; ++i) {
            const float sum = vx[i] + b;  // IEEE single, rounded to nearest, as on the device
            if (!(std::fabs((double)sum - row[i]) <= 0x1p-22 * std::fabs(row[i]))) return false;
        }
    }
    return true;
}

template <typename T>
spstd_status upload_field(spstd_ctx *ctx, const double *host, size_t off)
{
    if (sizeof(T) == 8) {
        SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(off), host, 8 * ctx->ntot, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        double *st = (double *)ctx->ptr(ctx->L.staging);
        SPSTD_CU(ctx, cudaMemcpyAsync(st, host, 8 * ctx->ntot, cudaMemcpyHostToDevice, ctx->stream));
        SPSTD_CU(ctx, Launch<T>::from_f64(st, (T *)ctx->ptr(off), ctx->ntot, ctx->stream));
    }
    return SPSTD_OK;
}
// Uploads state field f (0: psi_R, 1: psi_I) like upload_field and sums the
// squares of its FP64 values on the device into dout[4 + f]: half of
// N0 = dV sum(psi_R^2 + psi_I^2), the norm the divergence rule compares with,
// which the next spstd_energy_norm reads back with its own results.  The sum is
// taken from the FP64 values before any rounding to FP32, and no host pass
// over the arrays is needed.
template <typename T>
spstd_status upload_state_field(spstd_ctx *ctx, const double *host, int f)
{
    cudaStream_t s = ctx->stream;
    double *v64 = sizeof(T) == 8 ? (double *)ctx->ptr(ctx->L.psi[f]) : (double *)ctx->ptr(ctx->L.staging);
    double *part = (double *)ctx->ptr(ctx->L.partial);
    double *dout = (double *)ctx->ptr(ctx->L.dout);
    const int nb = (int)std::min<int64_t>(kPartials, (ctx->ntot + 255) / 256);
    SPSTD_CU(ctx, cudaMemcpyAsync(v64, host, 8 * ctx->ntot, cudaMemcpyHostToDevice, s));
    SPSTD_CU(ctx, Launch<double>::dot2(v64, v64, nullptr, nullptr, ctx->ntot, part, nb, s));
    SPSTD_CU(ctx, launch_sum_partials(part, nb, dout + 4 + f, s));
    if (sizeof(T) == 4) SPSTD_CU(ctx, Launch<T>::from_f64(v64, (T *)ctx->ptr(ctx->L.psi[f]), ctx->ntot, s));
    return SPSTD_OK;
}
// Enqueues the copy of a field to host FP64 values (through the FP64 staging
// field for FP32); the caller synchronises (check_device_status does).
template <typename T>
spstd_status download_field(spstd_ctx *ctx, const void *dev, double *host)
{
    if (sizeof(T) == 8) {
        SPSTD_CU(ctx, cudaMemcpyAsync(host, dev, 8 * ctx->ntot, cudaMemcpyDeviceToHost, ctx->stream));
    } else {
        double *st = (double *)ctx->ptr(ctx->L.staging);
        SPSTD_CU(ctx, Launch<T>::to_f64((const T *)dev, st, ctx->ntot, ctx->stream));
        SPSTD_CU(ctx, cudaMemcpyAsync(host, st, 8 * ctx->ntot, cudaMemcpyDeviceToHost, ctx->stream));
    }
    return SPSTD_OK;
}
}  // namespace

extern "C" {

spstd_status spstd_set_potential(spstd_ctx *ctx, const double *V)
{
    if (!ctx || !V) return SPSTD_EINVAL;
    double vmax = -INFINITY;
    for (int64_t i = 0; i < ctx->ntot; ++i) {
        if (!std::isfinite(V[i])) return fail(ctx, SPSTD_EINVAL, "V has a non-finite value");
        vmax = std::max(vmax, V[i]);
    }
    // kernel arguments name the tables (or not): replayed graphs are rebuilt,
    // and so are the descriptors of a batch the context belongs to
    drop_graph(ctx);
    batch_member_changed(ctx->batch);
    ctx->vsep = false;
    // the table form belongs to the reduce-add x passes
    if (ctx->cfg.precision == 32 && ctx->tma[0] && !ctx->cfg.v_field_only) {
        const int64_t n0 = ctx->cfg.n[0], rows = ctx->cfg.n[1] * ctx->cfg.n[2];
        std::vector<float> vx, vyz;
        if (separable_tables(V, n0, rows, vsep_rows_padded(rows), vx, vyz)) {
            float *dvx = (float *)ctx->ptr(ctx->L.vsep_x), *dvyz = (float *)ctx->ptr(ctx->L.vsep_yz);
            SPSTD_CU(ctx, cudaMemcpyAsync(dvx, vx.data(), 4 * vx.size(), cudaMemcpyHostToDevice, ctx->stream));
            SPSTD_CU(ctx, cudaMemcpyAsync(dvyz, vyz.data(), 4 * vyz.size(), cudaMemcpyHostToDevice, ctx->stream));
            // the V field holds the same FP32 sums, for every other pass
            SPSTD_CU(ctx, build_separable_v(dvx, dvyz, (float *)ctx->ptr(ctx->L.V), n0, rows, ctx->stream));
            SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
            ctx->vsep = true;
        }
    }
    spstd_status s = ctx->vsep ? SPSTD_OK
                     : ctx->cfg.precision == 32 ? upload_field<float>(ctx, V, ctx->L.V)
                                                : upload_field<double>(ctx, V, ctx->L.V);
    if (s != SPSTD_OK) return s;
    ctx->vmax = vmax;
    return set_dt(ctx, vmax);
}

spstd_status spstd_set_state(spstd_ctx *ctx, const double *psiR, const double *psiI)
{
    if (!ctx || !psiR || !psiI) return SPSTD_EINVAL;
    spstd_status s = ctx->cfg.precision == 32 ? upload_state_field<float>(ctx, psiR, 0)
                                              : upload_state_field<double>(ctx, psiR, 0);
    if (s != SPSTD_OK) return s;
    s = ctx->cfg.precision == 32 ? upload_state_field<float>(ctx, psiI, 1)
                                 : upload_state_field<double>(ctx, psiI, 1);
    if (s != SPSTD_OK) return s;
    SPSTD_CU(ctx, cudaMemsetAsync(ctx->ptr(ctx->L.counter), 0, 8, ctx->stream));
    ctx->steps_taken = 0;
    ctx->norm0_pending = true;
    return SPSTD_OK;
}

spstd_status spstd_get_state(spstd_ctx *ctx, double *psiR, double *psiI)
{
    if (!ctx || !psiR || !psiI) return SPSTD_EINVAL;
    // both fields are enqueued before the one synchronisation (the status read):
    // in stream order the staging field is not reused before its copy is done
    spstd_status s = ctx->cfg.precision == 32 ? download_field<float>(ctx, ctx->ptr(ctx->L.psi[0]), psiR)
                                              : download_field<double>(ctx, ctx->ptr(ctx->L.psi[0]), psiR);
    if (s != SPSTD_OK) return s;
    s = ctx->cfg.precision == 32 ? download_field<float>(ctx, ctx->ptr(ctx->L.psi[1]), psiI)
                                 : download_field<double>(ctx, ctx->ptr(ctx->L.psi[1]), psiI);
    if (s != SPSTD_OK) return s;
    return check_device_status(ctx);
}

spstd_status spstd_step(spstd_ctx *ctx, int64_t nsteps)
{
    if (!ctx || nsteps < 0) return SPSTD_EINVAL;
    NvtxRange r("spstd_step");
    if (nsteps == 0) return SPSTD_OK;
    return ctx->cfg.precision == 32 ? step_impl<float>(ctx, nsteps) : step_impl<double>(ctx, nsteps);
}

spstd_status spstd_probe(spstd_ctx *ctx, int p, double *re, double *im, int64_t cap, int64_t *len)
{
    if (!ctx || !re || !im || !len || cap < 0 || p < 0 || p >= ctx->cfg.n_probe) return SPSTD_EINVAL;
    *len = 0;
    if (ctx->steps_taken == 0) return fail(ctx, SPSTD_ENOTREADY, "no step recorded since set_state");
    const int64_t C = ctx->cfg.probe_capacity;
    const int64_t kept = std::min(ctx->steps_taken, C);
    const int64_t nout = std::min(kept, cap);
    const int64_t first = ctx->steps_taken - nout;  // global index of the first sample returned
    // only the samples returned are copied: one piece of the ring, or two where
    // it wraps; the status read below synchronises the stream for them
    std::vector<double2> row((size_t)nout);
    const double2 *ring = (const double2 *)ctx->ptr(ctx->L.ring) + (size_t)p * C;
    const int64_t i0 = nout > 0 ? first % C : 0;
    const int64_t n1 = std::min(nout, C - i0);
    if (n1 > 0)
        SPSTD_CU(ctx, cudaMemcpyAsync(row.data(), ring + i0, sizeof(double2) * n1, cudaMemcpyDeviceToHost, ctx->stream));
    if (nout > n1)
        SPSTD_CU(ctx, cudaMemcpyAsync(row.data() + n1, ring, sizeof(double2) * (nout - n1), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    spstd_status ds = check_device_status(ctx);
    if (ds != SPSTD_OK) return ds;
    for (int64_t i = 0; i < nout; ++i) {
        re[i] = row[i].x;
        im[i] = row[i].y;
    }
    *len = nout;
    return SPSTD_OK;
}

spstd_status spstd_spectrum(spstd_ctx *ctx, int p, int64_t nfft, int max_peaks, double thresh, int phase_correct,
                            double *E, double *amp, int *npeaks)
{
    if (!ctx || !E || !amp || !npeaks) return SPSTD_EINVAL;
    NvtxRange r("spstd_spectrum");
    *npeaks = 0;
    if (p < -1 || p >= ctx->cfg.n_probe || ctx->cfg.n_probe == 0) return fail(ctx, SPSTD_EINVAL, "bad probe");
    if (max_peaks < 1 || max_peaks > kMaxSpectrumPeaks) return fail(ctx, SPSTD_EINVAL, "max_peaks must be 1..64");
    if (!(thresh >= 0.0)) return fail(ctx, SPSTD_EINVAL, "thresh must be >= 0");
    const int64_t C = ctx->cfg.probe_capacity;
    const int64_t M = std::min(ctx->steps_taken, C);
    if (M < 2) return fail(ctx, SPSTD_ENOTREADY, "need at least 2 recorded steps");
    const int64_t maxn = effective_max_nfft(ctx->cfg);
    if (nfft <= 0) nfft = std::min(maxn, next_pow2(4 * M));
    if (!is_pow2(nfft) || nfft < M || nfft > maxn || nfft < 4)
        return fail(ctx, SPSTD_EINVAL, "nfft must be a power of two with M <= nfft <= max_nfft");
    SpectrumArgs a{};
    a.ring = (const double2 *)ctx->ptr(ctx->L.ring);
    a.n_probe = ctx->cfg.n_probe;
    a.p = p;
    a.cap = C;
    a.first_slot = (ctx->steps_taken - M) % C;
    a.M = M;
    a.nfft = nfft;
    a.max_nfft = maxn;
    a.max_peaks = max_peaks;
    a.thresh = thresh;
    a.scratch = ctx->ptr(ctx->L.spec);
    int np = 0;
    std::vector<double> th(max_peaks), am(max_peaks);
    a.h_npeaks = &np;
    a.h_theta = th.data();
    a.h_amp = am.data();
    SPSTD_CU(ctx, launch_spectrum(a, ctx->stream));
    spstd_status ds = check_device_status(ctx);
    if (ds != SPSTD_OK) return ds;
    std::vector<std::pair<double, double>> res;
    for (int i = 0; i < np; ++i) {
        double e = ctx->cfg.hbar * th[i] / ctx->dt;
        if (phase_correct) e = ctx->cfg.hbar * dispersion_inverse(ctx->m, ctx->c, ctx->d, ctx->s_star, th[i]) / ctx->dt;
        res.push_back({e, am[i]});
    }
    std::stable_sort(res.begin(), res.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    for (int i = 0; i < np; ++i) {
        E[i] = res[i].first;
        amp[i] = res[i].second;
    }
    *npeaks = np;
    return SPSTD_OK;
}

}  // extern "C"

namespace {
template <typename T>
spstd_status energy_norm_impl(spstd_ctx *ctx, double *norm, double *energy)
{
    cudaStream_t s = ctx->stream;
    T *pr = (T *)ctx->ptr(ctx->L.psi[0]);
    T *pi = (T *)ctx->ptr(ctx->L.psi[1]);
    T *tmp = (T *)ctx->ptr(ctx->L.tmp);
    double *part = (double *)ctx->ptr(ctx->L.partial);
    double *dout = (double *)ctx->ptr(ctx->L.dout);
    const int nb = (int)std::min<int64_t>(kPartials, (ctx->ntot + 255) / 256);
    const int tH = 2 * ctx->m;
    // sum psi_R^2 + psi_I^2
    SPSTD_CU(ctx, Launch<T>::dot2(pr, pr, pi, pi, ctx->ntot, part, nb, s));
    SPSTD_CU(ctx, launch_sum_partials(part, nb, dout + 0, s));
    // sum psi_R H psi_R
    SPSTD_CU(ctx, cudaMemsetAsync(tmp, 0, sizeof(T) * ctx->ntot, s));
    SPSTD_CU(ctx, enqueue_apply<T>(ctx, 0, 2, tH, 1.0, 0, s));
    SPSTD_CU(ctx, Launch<T>::dot2(pr, tmp, nullptr, nullptr, ctx->ntot, part, nb, s));
    SPSTD_CU(ctx, launch_sum_partials(part, nb, dout + 1, s));
    // sum psi_I H psi_I
    SPSTD_CU(ctx, cudaMemsetAsync(tmp, 0, sizeof(T) * ctx->ntot, s));
    SPSTD_CU(ctx, enqueue_apply<T>(ctx, 1, 2, tH, 1.0, 0, s));
    SPSTD_CU(ctx, Launch<T>::dot2(pi, tmp, nullptr, nullptr, ctx->ntot, part, nb, s));
    SPSTD_CU(ctx, launch_sum_partials(part, nb, dout + 2, s));
    // dout[4], dout[5]: the sums of squares of the state last set (N0)
    double h[6];
    SPSTD_CU(ctx, cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPSTD_CU(ctx, cudaStreamSynchronize(s));
    spstd_status ds = check_device_status(ctx);
    if (ds != SPSTD_OK) return ds;
    double dV = 1.0;
    for (int a = 0; a < ctx->cfg.dims; ++a) dV *= axis_spacing(ctx->cfg, a);
    if (ctx->norm0_pending) {
        ctx->norm0 = dV * (h[4] + h[5]);
        ctx->norm0_pending = false;
    }
    *norm = dV * h[0];
    *energy = dV * (h[1] + h[2]);
    if (!std::isfinite(*norm) || !std::isfinite(*energy)) return fail(ctx, SPSTD_EDIVERGED, "norm or energy is not finite");
    const double lim = ctx->cfg.norm_drift_limit;
    if (lim > 0 && ctx->norm0 > 0 && std::fabs(*norm / ctx->norm0 - 1.0) > lim) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "norm drifted by %.3e relative (limit %.1e): N = %.12g, N0 = %.12g",
                      *norm / ctx->norm0 - 1.0, lim, *norm, ctx->norm0);
        return fail(ctx, SPSTD_EDIVERGED, msg);
    }
    return SPSTD_OK;
}

template <typename T>
spstd_status apply_h_impl(spstd_ctx *ctx, int which, double *out)
{
    T *src = (T *)ctx->ptr(ctx->L.psi[which]);
    T *tmp = (T *)ctx->ptr(ctx->L.tmp);
    SPSTD_CU(ctx, cudaMemsetAsync(tmp, 0, sizeof(T) * ctx->ntot, ctx->stream));
    (void)src;
    SPSTD_CU(ctx, enqueue_apply<T>(ctx, which, 2, 2 * ctx->m, 1.0, 0, ctx->stream));
    spstd_status st = download_field<T>(ctx, tmp, out);
    return st != SPSTD_OK ? st : check_device_status(ctx);
}
}  // namespace

extern "C" {

spstd_status spstd_check_workspace(spstd_ctx *ctx, int *intact)
{
    if (!ctx || !intact) return SPSTD_EINVAL;
    *intact = 1;
    std::vector<unsigned char> g(kGuardBytes);
    for (int k = 0; k < ctx->L.n_guard; ++k) {
        SPSTD_CU(ctx, cudaMemcpyAsync(g.data(), ctx->ws + ctx->L.guard[k], kGuardBytes, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
        for (size_t i = 0; i < kGuardBytes; ++i) {
            if (g[i] != kGuardByte) {
                *intact = 0;
                char msg[96];
                std::snprintf(msg, sizeof(msg), "guard word %d (workspace offset %zu) overwritten", k,
                              ctx->L.guard[k] + i);
                ctx->err = msg;
                return SPSTD_OK;
            }
        }
    }
    return SPSTD_OK;
}

spstd_status spstd_energy_norm(spstd_ctx *ctx, double *norm, double *energy)
{
    if (!ctx || !norm || !energy) return SPSTD_EINVAL;
    NvtxRange r("spstd_energy_norm");
    return ctx->cfg.precision == 32 ? energy_norm_impl<float>(ctx, norm, energy)
                                    : energy_norm_impl<double>(ctx, norm, energy);
}

spstd_status spstd_apply_hamiltonian(spstd_ctx *ctx, int which, double *out)
{
    if (!ctx || !out || (which != 0 && which != 1)) return SPSTD_EINVAL;
    return ctx->cfg.precision == 32 ? apply_h_impl<float>(ctx, which, out) : apply_h_impl<double>(ctx, which, out);
}

}  // extern "C"

namespace {
template <typename T>
spstd_status profile_impl(spstd_ctx *ctx, int64_t nsteps, double *ms, int64_t *cnt)
{
    LaunchTimer timer;
    if (ctx->rk4) {
        for (int64_t i = 0; i < nsteps; ++i) SPSTD_CU(ctx, enqueue_rk4_step<T>(ctx, ctx->stream, &timer));
    } else if (resident_path(ctx)) {
        SPSTD_CU(ctx, launch_resident<T>(ctx, nsteps, &timer));
    } else {
        if (ctx->merge && nsteps > 0) {
            SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 0, 0, ctx->stream, &timer));
            SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 1, nsteps - 1, ctx->stream, &timer));
            SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 2, 0, ctx->stream, &timer));
        } else {
            SPSTD_CU(ctx, enqueue_steps<T>(ctx, nsteps, ctx->stream, &timer));
        }
    }
    ctx->steps_taken += nsteps;
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < SPSTD_KERNEL_KINDS; ++k) {
        ms[k] = 0.0;
        cnt[k] = 0;
    }
    for (size_t i = 0; i < timer.kind.size(); ++i) {
        float t = 0.f;
        SPSTD_CU(ctx, cudaEventElapsedTime(&t, timer.ev[2 * i], timer.ev[2 * i + 1]));
        ms[timer.kind[i]] += t;
        cnt[timer.kind[i]] += 1;
    }
    return SPSTD_OK;
}
}  // namespace

extern "C" {

spstd_status spstd_profile_steps(spstd_ctx *ctx, int64_t nsteps, double *ms, int64_t *cnt)
{
    if (!ctx || !ms || !cnt || nsteps < 0) return SPSTD_EINVAL;
    return ctx->cfg.precision == 32 ? profile_impl<float>(ctx, nsteps, ms, cnt)
                                    : profile_impl<double>(ctx, nsteps, ms, cnt);
}

spstd_status spstd_eigenstates_begin(spstd_ctx *ctx, int n_target, const double *E, int64_t window)
{
    if (!ctx || !E || window < 1) return SPSTD_EINVAL;
    if (n_target < 1 || n_target > ctx->cfg.max_eigenstates)
        return fail(ctx, SPSTD_EINVAL, "n_target must be 1..max_eigenstates");
    double theta[SPSTD_MAX_EIGENSTATES] = {0};
    for (int k = 0; k < n_target; ++k) {
        if (!std::isfinite(E[k])) return fail(ctx, SPSTD_EINVAL, "non-finite target energy");
        theta[k] = E[k] * ctx->dt / ctx->cfg.hbar;
    }
    SPSTD_CU(ctx, cudaMemsetAsync(ctx->ptr(ctx->L.eig_acc), 0, 16 * (size_t)n_target * ctx->ntot, ctx->stream));
    SPSTD_CU(ctx, cudaMemsetAsync(ctx->ptr(ctx->L.eig_step), 0, 16, ctx->stream));
    SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.eig_theta), theta, sizeof(theta), cudaMemcpyHostToDevice,
                                  ctx->stream));
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));  // theta lives on this stack
    ctx->eig_active = true;
    ctx->eig_n = n_target;
    ctx->eig_window = window;
    return SPSTD_OK;
}

spstd_status spstd_eigenstate_get(spstd_ctx *ctx, int k, int normalise, double *re, double *im, int64_t *samples)
{
    if (!ctx || !re || !im || k < 0 || k >= ctx->eig_n) return SPSTD_EINVAL;
    std::vector<double2> acc(ctx->ntot);
    int64_t n = 0;
    SPSTD_CU(ctx, cudaMemcpyAsync(acc.data(), (double2 *)ctx->ptr(ctx->L.eig_acc) + (size_t)k * ctx->ntot,
                                  sizeof(double2) * ctx->ntot, cudaMemcpyDeviceToHost, ctx->stream));
    SPSTD_CU(ctx, cudaMemcpyAsync(&n, ctx->ptr(ctx->L.eig_step), 8, cudaMemcpyDeviceToHost, ctx->stream));
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    // optional normalisation: sum |phi|^2 = 1, and the phase turned so that the
    // entry of largest modulus (the first such) is real and positive
    double ss = 0.0, amax = -1.0, cr = 1.0, ci = 0.0;
    int64_t jmax = 0;
    if (normalise) {
        for (int64_t p = 0; p < ctx->ntot; ++p) {
            const double a2 = acc[p].x * acc[p].x + acc[p].y * acc[p].y;
            ss += a2;
            if (a2 > amax) {
                amax = a2;
                jmax = p;
            }
        }
        if (ss > 0) {
            // multiply by conj(z_j)/|z_j| / sqrt(ss)
            const double aj = std::sqrt(amax), inv = 1.0 / std::sqrt(ss);
            cr = acc[jmax].x / aj * inv;
            ci = -acc[jmax].y / aj * inv;
        }
    }
    for (int64_t p = 0; p < ctx->ntot; ++p) {
        re[p] = acc[p].x * cr - acc[p].y * ci;
        im[p] = acc[p].x * ci + acc[p].y * cr;
    }
    if (normalise && ss > 0) im[jmax] = 0.0;
    if (samples) *samples = n;
    return SPSTD_OK;
}

spstd_status spstd_eigenstates_end(spstd_ctx *ctx)
{
    if (!ctx) return SPSTD_EINVAL;
    ctx->eig_active = false;
    return SPSTD_OK;
}

spstd_status spstd_get_dt(const spstd_ctx *ctx, double *dt)
{
    if (!ctx || !dt) return SPSTD_EINVAL;
    *dt = ctx->dt;
    return SPSTD_OK;
}

spstd_status spstd_separable_split(const double *V, int64_t nx, int64_t rows, float *vx, float *vyz,
                                   int *separable)
{
    if (!V || !vx || !vyz || !separable || nx < 1 || rows < 1) return SPSTD_EINVAL;
    std::vector<float> tx, tyz;
    const bool ok = separable_tables(V, nx, rows, rows, tx, tyz);
    std::memcpy(vx, tx.data(), sizeof(float) * nx);
    std::memcpy(vyz, tyz.data(), sizeof(float) * rows);
    *separable = ok ? 1 : 0;
    return SPSTD_OK;
}

spstd_status spstd_potential_separable(const spstd_ctx *ctx, int *separable)
{
    if (!ctx || !separable) return SPSTD_EINVAL;
    *separable = ctx->vsep ? 1 : 0;
    return SPSTD_OK;
}

spstd_status spstd_steps_taken(const spstd_ctx *ctx, int64_t *steps)
{
    if (!ctx || !steps) return SPSTD_EINVAL;
    *steps = ctx->steps_taken;
    return SPSTD_OK;
}

spstd_status spstd_get_coefficients(const spstd_ctx *ctx, int *m, double *c, double *d)
{
    if (!ctx || !m || !c || !d) return SPSTD_EINVAL;
    *m = ctx->m;
    for (int l = 0; l < ctx->m; ++l) {
        c[l] = ctx->c[l];
        d[l] = ctx->d[l];
    }
    return SPSTD_OK;
}

spstd_status spstd_launch_count(const spstd_ctx *ctx, int64_t nsteps, int64_t *launches)
{
    if (!ctx || !launches || nsteps < 0) return SPSTD_EINVAL;
    if (nsteps == 0) {
        *launches = 0;
    } else if (ctx->rk4) {
        // Runge-Kutta stage fields take the unfused passes
        *launches = nsteps * (8 * (ctx->cfg.dims + (ctx->long_x ? 2 : 0)) + 4 + (ctx->cfg.n_probe > 0 ? 1 : 0) +
                              (ctx->eig_active ? 1 : 0));
    } else if (ctx->eig_active) {
        *launches = nsteps * ((int64_t)ctx->hs.size() * apply_launches(ctx) + (ctx->cfg.n_probe > 0 ? 1 : 0) + 1);
    } else if (resident_path(ctx)) {
        *launches = 1;
    } else {
        if (ctx->merge) {
            // n (h - 1) + 1 half-stages; 2 (n - 1) + 1 probe launches
            const int64_t nh = (int64_t)ctx->hs.size();
            *launches = (nsteps * (nh - 1) + 1) * apply_launches(ctx) + (ctx->cfg.n_probe > 0 ? 2 * nsteps - 1 : 0);
        } else {
            // graph-replayed chunks of kGraphSteps, then the remainder
            const int64_t reps = nsteps >= kGraphSteps ? nsteps / kGraphSteps : 0;
            *launches = reps * launches_for_steps(ctx, kGraphSteps) +
                        launches_for_steps(ctx, nsteps - reps * kGraphSteps);
        }
    }
    return SPSTD_OK;
}

}  // extern "C"
