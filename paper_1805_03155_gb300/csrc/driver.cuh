// driver.cuh -- host-side internals of the C ABI, shared by its translation
// units (api.cu: contexts, stepping, reductions and spectra; batch.cu:
// batches and their autotuner; tune.cu: the per-context autotuner and
// schedule calls): the context structure, validation and workspace layout,
// FP64 host tables, tensor maps, and the enqueueing of half-stages and steps.
//
// The host code here computes only setup quantities (coefficient presets,
// the stability limit of Eq. 23-25, twiddle and k^2 tables, dispersion
// inversion of a few spectrum peaks); every step of the time integration,
// every reduction and every spectrum runs in the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/spstd.h"
#include "../../include/spstd_testing.h"
#include "dense_tc.h"
#include "launch.cuh"
#include "longline.h"
#include "pass_tma_launch.h"
#include "pass_xy.cuh"
#include "sched.h"
#include "spectrum.h"

using namespace spstd;

namespace spstd_host {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kPartials = 1024;        // blocks of the FP64 reductions (fixed: reproducible sums)
constexpr int kGraphSteps = 16;        // steps per captured graph (2D/3D)

struct HalfStage {
    int dst;      // field updated: 0 = psi_R, 1 = psi_I
    int table;    // multiplier table index
    double a;     // s coef dt hbar/2m*
    double bV;    // s coef dt/hbar
    double scale; // s coef dt (multiplies a dense operator that carries hbar/2m*)
};

// Guard words: kGuardBytes after every nonempty workspace region, filled with
// kGuardByte at creation; spstd_check_workspace reads them back, so that a
// kernel writing past the end of its region shows (a canary check, since the
// GPU sanitizer is not available to us).
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kMaxGuards = 48;

struct Layout {
    size_t psi[2], V, vsep_x, vsep_yz, tmp, staging, ring, counter, status, snap, partial, dout, tw[3], mult, dense[3], spec;
    size_t dense_tc[3];  // tensor-core form of a dense axis: D_hi then D_lo, [np][np] FP32 each
    size_t eig_acc, eig_theta, eig_step, rk[6], lscr, xy, total;
    size_t guard[kMaxGuards];
    int n_guard;
};

// Periodic lengths 3 * 2^k that the 2D/3D pass kernels transform with a
// radix-3 first stage (line_e and the plans of fft_line.cuh).
// A named NVTX range for the life of a scope (a no-op unless a profiler
// attaches): spstd_step, spstd_batch_step, spectra, reductions and tuning.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline bool is_radix3_len(int64_t n) { return n == 24 || n == 48 || n == 96 || n == 192 || n == 384; }

// An axis uses the FFT passes when it is periodic with a power-of-two length
// within the FFT limits, or (2D/3D grids) one of the radix-3 lengths;
// otherwise the dense operator (n <= SPSTD_MAX_DENSE_N).
inline bool axis_is_fft(const spstd_config &cfg, int a)
{
    const int64_t n = cfg.n[a];
    if (cfg.bc[a] != SPSTD_PERIODIC) return false;
    if ((n & (n - 1)) != 0) return cfg.dims > 1 && is_radix3_len(n);
    const int64_t lim = cfg.dims == 1 ? (cfg.precision == 32 ? 8192 : 4096) : 1024;
    return n >= 2 && n <= lim;
}

// The x axis of a periodic power-of-two length beyond the on-chip limit runs
// the four-step pass (up to 2^22 points).
inline bool axis_is_long(const spstd_config &cfg, int a)
{
    const int64_t n = cfg.n[a];
    return a == 0 && cfg.bc[a] == SPSTD_PERIODIC && (n & (n - 1)) == 0 && !axis_is_fft(cfg, a) && n <= kMaxLongN;
}

// 3D FP32 grids whose x and y axes both take the pipelined passes at the same
// length can run them as one fused launch (pass_xy.cuh).
inline bool xy_fusable(const spstd_config &cfg)
{
    auto tma_len = [](int64_t n) { return n == 64 || n == 128 || n == 256; };
    return cfg.precision == 32 && cfg.dims == 3 && cfg.n[0] == cfg.n[1] && tma_len(cfg.n[0]) &&
           cfg.bc[0] == SPSTD_PERIODIC && cfg.bc[1] == SPSTD_PERIODIC && cfg.n[2] >= 2;
}

// Entries of an axis in each multiplier row (the four-step pass computes its
// multipliers from the wrapped index instead).
inline int64_t table_len(const spstd_config &cfg, int a) { return a < cfg.dims && !axis_is_long(cfg, a) ? cfg.n[a] : 0; }

// Points per cell length: periodic L/n, Dirichlet L/(n+1), Neumann L/(n-1).
inline double axis_spacing(const spstd_config &cfg, int a)
{
    const double L = cfg.hi[a] - cfg.lo[a];
    const int64_t n = cfg.n[a];
    return cfg.bc[a] == SPSTD_DIRICHLET ? L / (double)(n + 1) : cfg.bc[a] == SPSTD_NEUMANN ? L / (double)(n - 1)
                                                                                           : L / (double)n;
}

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int64_t next_pow2(int64_t v)
{
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}
inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// ---- integrator coefficients (Eq. 17) ---------------------------------------
inline bool preset_coefficients(int id, int *m, double *c, double *d)
{
    switch (id) {
    case SPSTD_LEAPFROG:
        *m = 1;
        c[0] = 1.0;
        d[0] = 1.0;
        return true;
    case SPSTD_STRANG:
        *m = 2;
        c[0] = c[1] = 0.5;
        d[0] = 1.0;
        d[1] = 0.0;
        return true;
    case SPSTD_PAPER3: {
        // printed after Eq. 18, with d_l = c_{m-l+1}
        const double p[3] = {0.26833010, -0.18799162, 0.91966152};
        *m = 3;
        for (int l = 0; l < 3; ++l) {
            c[l] = p[l];
            d[l] = p[2 - l];
        }
        return true;
    }
    case SPSTD_FR4: {
        const double x = 1.0 / (2.0 - std::cbrt(2.0));
        const double cc[4] = {x / 2, (1 - x) / 2, (1 - x) / 2, x / 2};
        const double dd[4] = {x, 1 - 2 * x, x, 0.0};
        *m = 4;
        for (int l = 0; l < 4; ++l) {
            c[l] = cc[l];
            d[l] = dd[l];
        }
        return true;
    }
    case SPSTD_SUZUKI6: {
        const double p = 1.0 / (4.0 - std::cbrt(4.0));
        const double cc[6] = {p / 2, p, (1 - 3 * p) / 2, (1 - 3 * p) / 2, p, p / 2};
        const double dd[6] = {p, p, 1 - 4 * p, p, p, 0.0};
        *m = 6;
        for (int l = 0; l < 6; ++l) {
            c[l] = cc[l];
            d[l] = dd[l];
        }
        return true;
    }
    default:
        return false;
    }
}

// ---- stability (Eq. 23-25) ---------------------------------------------------
// Per-mode map of one step for s = w dt in stage order: each stage applies
// [[1, c s], [0, 1]] then [[1, 0], [-d s, 1]].
inline double step_trace(int m, const double *c, const double *d, double s)
{
    double m00 = 1, m01 = 0, m10 = 0, m11 = 1;
    for (int l = 0; l < m; ++l) {
        m00 += c[l] * s * m10;
        m01 += c[l] * s * m11;
        m10 -= d[l] * s * m00;
        m11 -= d[l] * s * m01;
    }
    return m00 + m11;
}

inline double stability_s_star(int m, const double *c, const double *d)
{
    const double h = 1e-4, smax = 64.0;
    double s = 0.0;
    while (s + h <= smax && std::fabs(step_trace(m, c, d, s + h)) <= 2.0) s += h;
    if (s + h > smax) return smax;
    double lo = s, hi = s + h;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (std::fabs(step_trace(m, c, d, mid)) <= 2.0) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Largest stable w dt of the configured scheme: the partitioned map's s*
// (Eq. 25), or 2 sqrt 2 for RK4 (|1 - is - s^2/2 + is^3/6 + s^4/24| <= 1 iff
// s^2 <= 8 on the imaginary axis).
inline double scheme_s_star(int preset, int m, const double *c, const double *d)
{
    if (preset == SPSTD_RK4) return 2.0 * std::sqrt(2.0);
    return stability_s_star(m, c, d);
}

// Phase advance per step of the mode with w dt = s. m = 0 is the classical
// Runge-Kutta scheme: its factor R(-is) = 1 - is - s^2/2 + is^3/6 + s^4/24 is
// not unimodular; the angle of exp(-i theta) is -arg R, taken in [0, pi].
inline double map_angle(int m, const double *c, const double *d, double s)
{
    if (m == 0) return std::fabs(std::atan2(s - s * s * s / 6.0, 1.0 - 0.5 * s * s + s * s * s * s / 24.0));
    double t = 0.5 * step_trace(m, c, d, s);
    t = std::min(1.0, std::max(-1.0, t));
    return std::acos(t);
}

// s with map_angle(s) = theta on the first increasing branch (Eq. 24/25: the
// eigenvalues of a det-1 map are exp(+-i theta), theta = arccos(tr/2)).
inline double dispersion_inverse(int m, const double *c, const double *d, double s_star, double theta)
{
    const double h = 1e-4;
    double top = 0.0;
    while (top + h <= s_star && map_angle(m, c, d, top + h) > map_angle(m, c, d, top)) top += h;
    if (theta >= map_angle(m, c, d, top)) return top;
    double lo = 0.0, hi = top;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (map_angle(m, c, d, mid) < theta) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

inline double w_max_of(const spstd_config &cfg, double vmax)
{
    // largest |k| per axis: pi n/L (periodic: the Nyquist mode; Dirichlet: the
    // n-th sine), pi (n-1)/L (Neumann: the (n-1)-th cosine)
    double w = 0.0;
    for (int a = 0; a < cfg.dims; ++a) {
        const double L = cfg.hi[a] - cfg.lo[a];
        const double kmax = kPi * (double)(cfg.bc[a] == SPSTD_NEUMANN ? cfg.n[a] - 1 : cfg.n[a]) / L;
        w += kmax * kmax;
    }
    return cfg.hbar / (2.0 * cfg.mass) * w + std::max(vmax, 0.0) / cfg.hbar;
}

// ---- validation and layout ---------------------------------------------------
inline spstd_status validate(const spstd_config *cfg, std::string *why, int *m, double *c, double *d)
{
    auto bad = [&](const char *w) {
        if (why) *why = w;
        return SPSTD_EINVAL;
    };
    if (!cfg) return bad("config is NULL");
    if (cfg->dims < 1 || cfg->dims > 3) return bad("dims must be 1, 2 or 3");
    if (cfg->precision != 32 && cfg->precision != 64) return bad("precision must be 32 or 64");
    for (int a = 0; a < 3; ++a) {
        if (a < cfg->dims) {
            if (cfg->bc[a] < SPSTD_PERIODIC || cfg->bc[a] > SPSTD_NEUMANN) return bad("unknown boundary condition");
            if (cfg->n[a] < 2) return bad("each used axis needs n >= 2");
            if (!(cfg->hi[a] > cfg->lo[a]) || !std::isfinite(cfg->hi[a] - cfg->lo[a])) return bad("box needs hi > lo");
        } else if (cfg->n[a] != 1) {
            return bad("unused axes must have n = 1");
        }
    }
    for (int a = 0; a < cfg->dims; ++a) {
        if (!axis_is_fft(*cfg, a) && !axis_is_long(*cfg, a) && cfg->n[a] > SPSTD_MAX_DENSE_N) {
            if (why)
                *why = "axis not supported: FFT axes are periodic powers of two (x <= 4194304; y, z <= 1024) "
                       "or, in 2D/3D, 3 * 2^k for 24 <= n <= 384; other axes need n <= 256";
            return SPSTD_EUNSUPPORTED;
        }
    }
    if (!(cfg->hbar > 0) || !(cfg->mass > 0)) return bad("hbar and mass must be > 0");
    if (cfg->preset == SPSTD_CUSTOM) {
        if (cfg->m < 1 || cfg->m > SPSTD_MAX_STAGES) return bad("custom integrator needs 1 <= m <= 8");
        *m = cfg->m;
        for (int l = 0; l < cfg->m; ++l) {
            if (!std::isfinite(cfg->c[l]) || !std::isfinite(cfg->d[l])) return bad("non-finite coefficient");
            c[l] = cfg->c[l];
            d[l] = cfg->d[l];
        }
    } else if (cfg->preset == SPSTD_RK4) {
        *m = 0;  // not a partitioned scheme: no c_l, d_l
    } else if (!preset_coefficients(cfg->preset, m, c, d)) {
        return bad("unknown integrator preset");
    }
    int nh = 0;
    for (int l = 0; l < *m; ++l) nh += (c[l] != 0.0) + (d[l] != 0.0);
    if (nh == 0 && cfg->preset != SPSTD_RK4) return bad("all integrator coefficients are zero");
    if (nh > kMaxHalfStages) return bad("too many nonzero coefficients");
    if (cfg->n_probe < 0 || cfg->n_probe > SPSTD_MAX_PROBES) return bad("n_probe must be 0..16");
    const int64_t ntot = cfg->n[0] * cfg->n[1] * cfg->n[2];
    for (int q = 0; q < cfg->n_probe; ++q)
        if (cfg->probe_idx[q] < 0 || cfg->probe_idx[q] >= ntot) return bad("probe index outside the grid");
    if (cfg->probe_capacity < 1) return bad("probe_capacity must be >= 1");
    if (cfg->max_nfft > 0 && (!is_pow2(cfg->max_nfft) || cfg->max_nfft < 4)) return bad("max_nfft must be a power of two >= 4");
    if (cfg->max_eigenstates < 0 || cfg->max_eigenstates > SPSTD_MAX_EIGENSTATES) return bad("max_eigenstates must be 0..4");
    if (!std::isfinite(cfg->dt)) return bad("dt is not finite");
    if (std::isnan(cfg->norm_drift_limit)) return bad("norm_drift_limit is NaN");
    return SPSTD_OK;
}

inline int64_t effective_max_nfft(const spstd_config &cfg)
{
    if (cfg.max_nfft > 0) return cfg.max_nfft;
    return std::max<int64_t>(4, next_pow2(4 * cfg.probe_capacity));
}

inline int64_t vsep_rows_padded(int64_t rows) { return (rows + 127) / 128 * 128; }

// A dense axis of an FP32 2D/3D grid with 32..128 points runs on the tensor
// cores (dense_tc.h); 1D grids keep the resident dense kernel.
inline bool dense_tc_axis(const spstd_config &cfg, int a)
{
    return a < cfg.dims && cfg.dims >= 2 && cfg.precision == 32 && !axis_is_fft(cfg, a) && !axis_is_long(cfg, a) &&
           dense_tc_eligible(cfg.n[a]);
}

inline Layout make_layout(const spstd_config &cfg, int m)
{
    Layout L{};
    const int64_t ntot = cfg.n[0] * cfg.n[1] * cfg.n[2];
    const size_t es = cfg.precision == 32 ? 4 : 8;
    size_t off = 0;
    L.n_guard = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes);
        if (bytes > 0 && L.n_guard < kMaxGuards) {
            L.guard[L.n_guard++] = off;
            off += kGuardBytes;
        }
        return o;
    };
    L.psi[0] = take(es * ntot);
    L.psi[1] = take(es * ntot);
    L.V = take(es * ntot);
    // separable-potential tables of the FP32 x pass: vx, then vyz padded with
    // zeros to whole x tiles (at most 128 rows each)
    const bool sep = cfg.precision == 32 && cfg.dims >= 2;
    L.vsep_x = take(sep ? 4 * (size_t)cfg.n[0] : 0);
    L.vsep_yz = take(sep ? 4 * (size_t)vsep_rows_padded(cfg.n[1] * cfg.n[2]) : 0);
    L.tmp = take(es * ntot);
    L.staging = take(cfg.precision == 32 ? 8 * ntot : 0);
    L.ring = take(16 * (size_t)std::max(cfg.n_probe, 1) * cfg.probe_capacity);
    L.counter = take(8);
    L.status = take(8);
    L.snap = take(16 * SPSTD_MAX_PROBES);
    L.partial = take(8 * kPartials);
    L.dout = take(8 * 8);
    int64_t sum_n = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t ntw = a < cfg.dims ? cfg.n[a] : 0;
        if (a < cfg.dims && axis_is_long(cfg, a)) {
            int N1, N2;
            long_split(cfg.n[a], &N1, &N2);
            ntw = N1 + 2 * (int64_t)N2;  // W_N1, W_N2, W_N[k < N2]
        }
        L.tw[a] = take(2 * es * ntw);
        sum_n += table_len(cfg, a);
    }
    L.mult = take(es * (size_t)(2 * m + 2) * sum_n);  // rows: c_l, d_l, H, merged boundary
    for (int a = 0; a < 3; ++a)
        L.dense[a] = take(a < cfg.dims && !axis_is_fft(cfg, a) && !axis_is_long(cfg, a)
                              ? es * (size_t)cfg.n[a] * cfg.n[a] : 0);
    for (int a = 0; a < 3; ++a)
        L.dense_tc[a] = take(dense_tc_axis(cfg, a) ? 2 * 4 * (size_t)dense_tc_pad(cfg.n[a]) * dense_tc_pad(cfg.n[a]) : 0);
    L.spec = take(spectrum_scratch_bytes(effective_max_nfft(cfg), cfg.probe_capacity));
    L.eig_acc = take(16 * (size_t)cfg.max_eigenstates * ntot);
    L.eig_theta = take(8 * SPSTD_MAX_EIGENSTATES);
    L.eig_step = take(16);  // int64 step, unsigned completion count
    for (int k = 0; k < 6; ++k) L.rk[k] = take(cfg.preset == SPSTD_RK4 ? es * ntot : 0);  // t, h, acc (R, I)
    // four-step scratch: one complex line per pair of x lines
    L.lscr = take(axis_is_long(cfg, 0) ? 2 * es * (size_t)((cfg.n[1] * cfg.n[2] + 1) / 2) * cfg.n[0] : 0);
    // fused x-y pass counters: ticket/claim words, then per plane y tiles done and x tiles seen
    L.xy = take(xy_fusable(cfg) ? 4 * (size_t)(4 + 2 * cfg.n[2]) : 0);
    L.total = off;
    return L;
}

}  // namespace spstd_host

using namespace spstd_host;

struct spstd_ctx {
    spstd_config cfg;
    int m = 0;
    double c[SPSTD_MAX_STAGES] = {0}, d[SPSTD_MAX_STAGES] = {0};
    double s_star = 0, dt = 0, vmax = 0;
    bool dt_auto = false;
    int64_t ntot = 0, sum_n = 0;
    Layout L{};
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<HalfStage> hs;
    int64_t steps_taken = 0;
    double norm0 = 0.0;  // norm of the state last set (divergence rule)
    bool norm0_pending = false;  // its two FP64 sums wait in dout[4], dout[5] on the device
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    // pipelined FP32 passes: tensor maps [field: psi_R, psi_I, tmp][view: x, y, z]
    // default (reduce-add) passes: tma[axis]; x view of psi_R, psi_I, tmp, V;
    // y and z views of the fields, with the boxes of pass_tmared.cuh
    bool tma[3] = {false, false, false};
    CUtensorMap xrmap[4];
    // x pass with per-warp tiles (schedule 6): eligible, maps (psi_R, psi_I, tmp, V)
    bool xw_ok = false;
    CUtensorMap xwmap[4];
    // RK4 comparison scheme: reduce-add maps of its stage fields t_R, t_I, h_R,
    // h_I (fields 3..6) in the x, y and z views, so its H applications take the
    // TMA passes too
    bool rk_tma[3] = {false, false, false};
    CUtensorMap rkmap[4][3];
    CUtensorMap srmap[3][2];
    // stored-tile passes (schedule 5, fused x-y): tma_st[axis]; [field][view]
    bool tma_st[3] = {false, false, false};
    CUtensorMap tmap[3][3];
    spstd_batch *batch = nullptr;  // batch this context is a member of
    bool dense[3] = {false, false, false};  // axis applies the dense operator
    bool long_x = false;                    // x axis runs the four-step pass
    int N1 = 0, N2 = 0;                     // its split N = N1 N2
    int64_t tab_off[3] = {0, 0, 0};         // axis offsets within a multiplier row
    int sched[3] = {0, 0, 0};               // pass schedule per axis (sched.h)
    bool fuse_xy = false;                   // x and y passes as one launch (when both are schedule 0)
    // fused x-y reduce-add pass for nx = ny in {32, 64}: eligible, in use, maps
    // (psi_R, psi_I, tmp, V in the unit view)
    bool fxy_ok = false, fxy_on = false;
    CUtensorMap fxmap[4];
    // the potential is separable, V = vx(x) + vyz(y, z): the reduce-add x pass
    // rebuilds the V term from the tables at L.vsep_x / L.vsep_yz
    bool vsep = false;
    // step-boundary merge of the last and first half-stages (same field)
    bool merge = false;
    HalfStage merged{};
    double merge_alpha = 0.0;  // c_last / (c_last + c_first)
    // eigenstate accumulation window
    bool rk4 = false;  // classical Runge-Kutta comparison scheme
    bool eig_active = false;
    int eig_n = 0;
    int64_t eig_window = 0;

    void *ptr(size_t off) { return ws + off; }
    // fields: 0 psi_R, 1 psi_I, 2 scratch, 3..8 Runge-Kutta t_R, t_I, h_R, h_I, acc_R, acc_I
    size_t field_off(int f) const { return f == 0 ? L.psi[0] : f == 1 ? L.psi[1] : f == 2 ? L.tmp : L.rk[f - 3]; }
};

namespace spstd_host {

inline spstd_status fail(spstd_ctx *ctx, spstd_status s, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return s;
}
inline spstd_status cuda_fail(spstd_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, SPSTD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define SPSTD_CU(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Reads the device status word after a synchronisation: a kernel that gave up
// a bounded wait leaves kStatusTimeout there.
inline spstd_status check_device_status(spstd_ctx *ctx)
{
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, ctx->ptr(ctx->L.status), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (st != 0) {
        // a timed-out fused pass may leave its counters mid-count: clear them with the status
        if (xy_fusable(ctx->cfg))
            cudaMemsetAsync(ctx->ptr(ctx->L.xy), 0, 4 * (size_t)(4 + 2 * ctx->cfg.n[2]), ctx->stream);
        cudaMemsetAsync(ctx->ptr(ctx->L.status), 0, sizeof(int), ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        return fail(ctx, SPSTD_ETIMEOUT, "a device wait timed out (status word set by a pass kernel)");
    }
    return SPSTD_OK;
}

// A batch's descriptors hold its members' dt-derived coefficients and table
// pointers: a member whose potential (hence dt or table form) changes makes the
// batch rebuild them before its next step (batch.cu).
void batch_member_changed(spstd_batch *b);

inline void drop_graph(spstd_ctx *ctx)
{
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
}

// k^2 of DFT index j on an n-point axis of period L (wrapped index, Eq. 8).
inline double k2_of(int64_t j, int64_t n, double L, int nyquist_zero)
{
    if (nyquist_zero && n % 2 == 0 && j == n / 2) return 0.0;
    const int64_t w = (j <= n / 2) ? j : j - n;
    const double k = 2.0 * kPi * (double)w / L;
    return k * k;
}

// Spectral second-derivative operator of one axis as a dense n x n matrix
// (row-major; symmetric except for Neumann walls, whose DCT-I weights the wall
// points by one half), in FP64: the periodic operator F^-1 k^2 F of the
// line's extension (itself for periodic axes; the odd extension over twice
// the box for Dirichlet walls, the even one for Neumann walls, Section 2.2)
// folded back onto the n grid points.  A[r] = (1/P) sum_q k_q^2 cos(2 pi q r/P)
// is the circulant of the extended line of P points and period Lp.
inline std::vector<double> dense_operator(const spstd_config &cfg, int axis)
{
    const int64_t n = cfg.n[axis];
    const int bc = cfg.bc[axis];
    const double L = cfg.hi[axis] - cfg.lo[axis];
    const int64_t P = bc == SPSTD_DIRICHLET ? 2 * (n + 1) : bc == SPSTD_NEUMANN ? 2 * (n - 1) : n;
    const double Lp = bc == SPSTD_PERIODIC ? L : 2.0 * L;
    std::vector<double> A(P, 0.0);
    for (int64_t r = 0; r < P; ++r) {
        double acc = 0.0;
        for (int64_t q = 0; q < P; ++q)
            acc += k2_of(q, P, Lp, bc == SPSTD_PERIODIC ? cfg.nyquist_zero : 0) *
                   std::cos(2.0 * kPi * (double)((q * r) % P) / (double)P);
        A[r] = acc / (double)P;
    }
    auto circ = [&](int64_t d) { return A[((d % P) + P) % P]; };
    std::vector<double> D((size_t)n * n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double v;
            if (bc == SPSTD_DIRICHLET) {
                // f_j sits at p = j+1 (+) and p = P-1-j (-); output i at p = i+1
                v = circ((i + 1) - (j + 1)) - circ((i + 1) - (P - 1 - j));
            } else if (bc == SPSTD_NEUMANN) {
                // f_j sits at p = j and, for interior j, also at p = P-j
                v = circ(i - j);
                if (j > 0 && j < n - 1) v += circ(i - (P - j));
            } else {
                v = circ(i - j);
            }
            D[(size_t)i * n + j] = v;
        }
    }
    return D;
}

// The factor a of multiplier row t (the row holds a k^2/N): c_l dt hbar/2m*
// (row 2l), -d_l dt hbar/2m* (row 2l+1), hbar^2/2m* (H), merged boundary.
inline double table_a(const spstd_ctx *ctx, int t)
{
    const spstd_config &cfg = ctx->cfg;
    const int m = ctx->m;
    if (t == 2 * m + 1) return ctx->merge ? ctx->merged.a : 0.0;
    if (t == 2 * m) return cfg.hbar * cfg.hbar / (2.0 * cfg.mass);
    return (t & 1) ? -ctx->d[t / 2] * ctx->dt * cfg.hbar / (2.0 * cfg.mass)
                   : +ctx->c[t / 2] * ctx->dt * cfg.hbar / (2.0 * cfg.mass);
}

// x rounded to TF32 (FP32 with the 13 low mantissa bits zero: the bits a
// TF32 MMA reads), to nearest, ties away from zero, via FP32.
inline double tf32_of(double x)
{
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    std::memcpy(&f, &u, 4);
    return f;
}

template <typename T>
spstd_status upload_tables(spstd_ctx *ctx)
{
    const spstd_config &cfg = ctx->cfg;
    // twiddles W_N[k] = exp(-2 pi i k/N), FP64 then rounded
    std::vector<std::vector<T>> tws(3);
    for (int a = 0; a < cfg.dims; ++a) {
        std::vector<T> &tw = tws[a];
        // W_n[k] = exp(-2 pi i k/n), k < count, appended
        auto append = [&](int64_t n, int64_t count) {
            for (int64_t k = 0; k < count; ++k) {
                const double ang = 2.0 * kPi * (double)k / (double)n;
                tw.push_back((T)std::cos(ang));
                tw.push_back((T)(-std::sin(ang)));
            }
        };
        if (a == 0 && ctx->long_x) {
            append(ctx->N1, ctx->N1);
            append(ctx->N2, ctx->N2);
            append(cfg.n[0], ctx->N2);
        } else {
            append(cfg.n[a], cfg.n[a]);
        }
        SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.tw[a]), tw.data(), sizeof(T) * tw.size(), cudaMemcpyHostToDevice,
                                      ctx->stream));
    }
    // per half-stage (and H) multipliers a k_d^2(n)/N_d, FP64 then rounded
    const int ntab = 2 * ctx->m + 2;
    std::vector<double> a_of(ntab, 0.0);
    for (int t = 0; t < ntab; ++t) a_of[t] = table_a(ctx, t);
    std::vector<T> mult((size_t)ntab * ctx->sum_n);
    for (int t = 0; t < ntab; ++t) {
        for (int a = 0; a < cfg.dims; ++a) {
            const int64_t n = table_len(cfg, a);
            const double L = cfg.hi[a] - cfg.lo[a];
            for (int64_t j = 0; j < n; ++j)
                mult[(size_t)t * ctx->sum_n + ctx->tab_off[a] + j] =
                    (T)(a_of[t] * k2_of(j, n, L, cfg.nyquist_zero) / (double)n);
        }
    }
    SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.mult), mult.data(), sizeof(T) * mult.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    // dense operators of the non-FFT axes, times hbar/2m*
    std::vector<std::vector<T>> dense(3);
    std::vector<std::vector<float>> tc(3);
    for (int a = 0; a < cfg.dims; ++a) {
        if (!ctx->dense[a]) continue;
        // stored transposed (column-major), so that the threads of a line, one
        // output point each, read consecutive entries
        std::vector<double> D = dense_operator(cfg, a);
        const int64_t n = cfg.n[a];
        dense[a].resize(D.size());
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                dense[a][(size_t)j * n + i] = (T)(cfg.hbar / (2.0 * cfg.mass) * D[(size_t)i * n + j]);
        SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.dense[a]), dense[a].data(), sizeof(T) * dense[a].size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
        if (dense_tc_axis(cfg, a)) {
            // tensor-core form: rows i, columns j, zero padded to np, in the
            // MMA operand layout; each entry split in FP64 as hi = TF32(D),
            // lo = TF32(D - hi)
            const int np = dense_tc_pad(n);
            std::vector<float> &t = tc[a];
            t.assign(2 * (size_t)np * np, 0.f);
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = 0; j < n; ++j) {
                    const double d = cfg.hbar / (2.0 * cfg.mass) * D[(size_t)i * n + j];
                    const double hi = tf32_of(d);
                    const size_t o = dense_tc_offset((int)i, (int)j, np);
                    t[o] = (float)hi;
                    t[(size_t)np * np + o] = (float)tf32_of(d - hi);
                }
            SPSTD_CU(ctx, cudaMemcpyAsync(ctx->ptr(ctx->L.dense_tc[a]), t.data(), sizeof(float) * t.size(),
                                          cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    // the host vectors die here: wait until the copies have read them
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return SPSTD_OK;
}

// cuTensorMapEncodeTiled from the driver, without linking libcuda.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3D FP32 tensor map over a field viewed as dims (d0, d1, d2), x fastest, with
// the given box; out-of-range box elements load as zero and are not stored.
inline bool encode_map(CUtensorMap *m, void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
                uint32_t b2, bool swizzle128)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * sizeof(float), d0 * d1 * sizeof(float)};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Planes per tile of the reduce-add strided pass of axis ax (1 for the x pass).
inline int red_planes(const int64_t *n, int ax)
{
    if (ax == 0) return 1;
    return tmared_planes((int)n[ax], tmared_pairs((int)n[ax], n[0]), ax == 1 ? n[2] : n[1]);
}

// 4D FP32 tensor map (dims d[0] fastest; strides of dims 1..3 in elements)
// with the given box; out-of-range box elements load as zero and are not
// written back.
inline bool encode_map4(CUtensorMap *m, void *base, const uint64_t *d, const uint64_t *stride, const uint32_t *box)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {d[0], d[1], d[2], d[3]};
    const cuuint64_t strides[3] = {stride[0] * sizeof(float), stride[1] * sizeof(float), stride[2] * sizeof(float)};
    const cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of the reduce-add passes (pass_tmared.cuh): the line axis of length N
// is split as (L1, L2) = (min(N, 256), N / L1) so that no box dimension
// exceeds 256.  v = 0: x view (x_lo, x_hi, row, 1); v = 1: y view (x, y_lo,
// y_hi, z); v = 2: z view (x, y, z_lo, z_hi).  Strided boxes span
// tmared_planes() planes of the outer axis.
// x view (x_lo, x_hi, row, 1) with a box of `rows` rows.
inline bool encode_x_rows_map(CUtensorMap *m, void *base, const int64_t *n, int rows)
{
    const uint64_t n0 = n[0], n1 = n[1], n2 = n[2];
    const uint64_t L1 = n0 < 256 ? n0 : 256, L2 = n0 / L1;
    const uint64_t d[4] = {L1, L2, n1 * n2, 1}, st[3] = {L1, n0, n0 * n1 * n2};
    const uint32_t box[4] = {(uint32_t)L1, (uint32_t)L2, (uint32_t)rows, 1};
    return encode_map4(m, base, d, st, box);
}

inline bool encode_red_map(CUtensorMap *m, void *base, const int64_t *n, int v)
{
    const uint64_t n0 = n[0], n1 = n[1], n2 = n[2];
    const uint64_t N = (uint64_t)n[v], L1 = N < 256 ? N : 256, L2 = N / L1;
    if (v == 0) {
        const uint64_t d[4] = {L1, L2, n1 * n2, 1}, st[3] = {L1, n0, n0 * n1 * n2};
        const uint32_t box[4] = {(uint32_t)L1, (uint32_t)L2, (uint32_t)tmared_rows_x((int)N), 1};
        return encode_map4(m, base, d, st, box);
    }
    const int P = tmared_pairs((int)N, (int64_t)n0);
    const uint32_t cols = 2u * (uint32_t)P, K = (uint32_t)red_planes(n, v);
    if (v == 1) {
        const uint64_t d[4] = {n0, L1, L2, n2}, st[3] = {n0, n0 * L1, n0 * n1};
        const uint32_t box[4] = {cols, (uint32_t)L1, (uint32_t)L2, K};
        return encode_map4(m, base, d, st, box);
    }
    const uint64_t d[4] = {n0, n1, L1, L2}, st[3] = {n0, n0 * n1, n0 * n1 * L1};
    const uint32_t box[4] = {cols, K, (uint32_t)L1, (uint32_t)L2};
    return encode_map4(m, base, d, st, box);
}

// Enables the pipelined passes for FP32 axes of 32..512 points.
inline void setup_tma(spstd_ctx *ctx)
{
    const spstd_config &cfg = ctx->cfg;
    if (cfg.precision != 32 || cfg.dims < 2) return;
    const uint64_t n0 = cfg.n[0], n1 = cfg.n[1], n2 = cfg.n[2];
    auto stored_ok = [](int64_t n) { return n == 64 || n == 128 || n == 256; };
    for (int v = 0; v < cfg.dims; ++v) {
        if (ctx->dense[v]) continue;
        // stored-tile passes (schedule 5 and the fused x-y pass): 32-row / 32-column boxes
        bool ok = stored_ok(cfg.n[v]);
        for (int f = 0; f < 3 && ok; ++f) {
            void *base = ctx->ptr(ctx->field_off(f));
            if (v == 0) ok = encode_map(&ctx->tmap[f][0], base, n0, n1 * n2, 1, (uint32_t)n0, tma_rows_per_tile(), 1, false);
            if (v == 1) ok = encode_map(&ctx->tmap[f][1], base, n0, n1, n2, tma_cols_per_tile(), (uint32_t)n1, 1, false);
            if (v == 2) ok = encode_map(&ctx->tmap[f][2], base, n0, n1, n2, tma_cols_per_tile(), 1, (uint32_t)n2, false);
        }
        ctx->tma_st[v] = ok;
        // reduce-add passes (the default): boxes sized per line length
        ok = tmared_eligible(cfg.n[v]) && (v == 0 || tmared_pairs((int)cfg.n[v], cfg.n[0]) > 0);
        for (int f = 0; f < 4 && ok; ++f) {
            void *base = f < 3 ? ctx->ptr(ctx->field_off(f)) : ctx->ptr(ctx->L.V);
            if (v == 0) ok = encode_red_map(&ctx->xrmap[f], base, cfg.n, 0);
            else if (f < 3) ok = encode_red_map(&ctx->srmap[f][v - 1], base, cfg.n, v);
        }
        ctx->tma[v] = ok;
        // the RK4 stage fields on the same boxes
        if (ok && ctx->rk4) {
            bool okr = true;
            for (int f = 3; f <= 6 && okr; ++f)
                okr = encode_red_map(&ctx->rkmap[f - 3][v], ctx->ptr(ctx->field_off(f)), cfg.n, v);
            ctx->rk_tma[v] = okr;
        }
        // per-warp x tiles (schedule 6)
        if (v == 0 && ok && xwarp_eligible(cfg.n[0])) {
            bool okw = true;
            for (int f = 0; f < 4 && okw; ++f)
                okw = encode_x_rows_map(&ctx->xwmap[f], f < 3 ? ctx->ptr(ctx->field_off(f)) : ctx->ptr(ctx->L.V),
                                        cfg.n, xwarp_rows((int)cfg.n[0]));
            ctx->xw_ok = okw;
        }
    }
    // fused x-y pass: unit view (x, y, 1, z), box (N, N, 1, K)
    if (fxy_eligible(cfg.n, cfg.dims) && ctx->tma[0] && ctx->tma[1]) {
        bool ok = true;
        const uint64_t d[4] = {n0, n1, 1, n2}, st[3] = {n0, n0 * n1, n0 * n1};
        const uint32_t box[4] = {(uint32_t)n0, (uint32_t)n1, 1, (uint32_t)fxy_planes((int)n0)};
        for (int f = 0; f < 4 && ok; ++f)
            ok = encode_map4(&ctx->fxmap[f], f < 3 ? ctx->ptr(ctx->field_off(f)) : ctx->ptr(ctx->L.V), d, st, box);
        ctx->fxy_ok = ok;
        ctx->fxy_on = ok;
    }
}

inline spstd_status set_dt(spstd_ctx *ctx, double vmax)
{
    const double wmax = w_max_of(ctx->cfg, vmax);
    const double dt_max = ctx->s_star / wmax;
    double dt = ctx->dt_auto ? 0.5 * dt_max : ctx->cfg.dt;
    if (!ctx->dt_auto && dt > dt_max)
        return fail(ctx, SPSTD_EUNSTABLE, "dt is above the stability limit s*/w_max = " + std::to_string(dt_max));
    const bool changed = dt != ctx->dt;
    ctx->dt = dt;
    ctx->hs.clear();
    for (int l = 0; l < ctx->m; ++l) {
        const double k = ctx->cfg.hbar / (2.0 * ctx->cfg.mass);
        if (ctx->c[l] != 0.0)
            ctx->hs.push_back({0, 2 * l, ctx->c[l] * dt * k, ctx->c[l] * dt / ctx->cfg.hbar, ctx->c[l] * dt});
        if (ctx->d[l] != 0.0)
            ctx->hs.push_back({1, 2 * l + 1, -ctx->d[l] * dt * k, -ctx->d[l] * dt / ctx->cfg.hbar, -ctx->d[l] * dt});
    }
    ctx->merge = false;
    if (!ctx->cfg.unmerged_steps && ctx->hs.size() >= 2 && ctx->hs.front().dst == ctx->hs.back().dst) {
        const HalfStage &f = ctx->hs.front(), &l = ctx->hs.back();
        if (f.scale + l.scale != 0.0) {
            ctx->merge = true;
            ctx->merged = {f.dst, 2 * ctx->m + 1, f.a + l.a, f.bV + l.bV, f.scale + l.scale};
            ctx->merge_alpha = l.scale / (f.scale + l.scale);
        }
    }
    if (changed || ctx->gexec == nullptr) {
        drop_graph(ctx);
        spstd_status s = ctx->cfg.precision == 32 ? upload_tables<float>(ctx) : upload_tables<double>(ctx);
        if (s != SPSTD_OK) return s;
    }
    return SPSTD_OK;
}

// dst += a sum_d L_d src + bV V src  (table: multiplier set, use_V: add the V term)
// Optional per-launch timing: when set, an event pair brackets every launch.
struct LaunchTimer {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    cudaError_t begin(cudaStream_t s)
    {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
        return cudaEventRecord(e, s);
    }
    cudaError_t end(cudaStream_t s, int k)
    {
        kind.push_back(k);
        return begin(s);
    }
    ~LaunchTimer()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

#define SPSTD_TIMED(timer, s, k, call)                  \
    do {                                                \
        if (timer) {                                    \
            cudaError_t e0_ = (timer)->begin(s);        \
            if (e0_ != cudaSuccess) return e0_;         \
        }                                               \
        cudaError_t e1_ = (call);                       \
        if (e1_ != cudaSuccess) return e1_;             \
        if (timer) {                                    \
            cudaError_t e2_ = (timer)->end(s, k);       \
            if (e2_ != cudaSuccess) return e2_;         \
        }                                               \
    } while (0)

template <typename T>
T *field_ptr(spstd_ctx *ctx, int f)
{
    return (T *)ctx->ptr(ctx->field_off(f));
}

// Factor of a dense operator (which carries hbar/2m*) for multiplier set
// `table`: s coef dt for a half-stage, hbar for H (row 2m).
inline double table_scale(const spstd_ctx *ctx, int table)
{
    if (table == 2 * ctx->m + 1) return ctx->merged.scale;
    if (table >= 2 * ctx->m) return ctx->cfg.hbar;
    const int l = table / 2;
    return (table & 1) ? -ctx->d[l] * ctx->dt : ctx->c[l] * ctx->dt;
}

// Whether an H-apply between psi_R, psi_I and the scratch field runs x and y as one launch.
inline bool fused_active(const spstd_ctx *ctx) { return ctx->fuse_xy && ctx->sched[0] == 0 && ctx->sched[1] == 0; }

// Whether H-applies between the state fields run x and y as the fused reduce-add pass.
inline bool fxy_active(const spstd_ctx *ctx)
{
    return !fused_active(ctx) && ctx->fxy_ok && ctx->fxy_on && ctx->sched[0] == 0 && ctx->sched[1] == 0;
}

// dst += a sum_d L_d src + bV V src for fields fsrc -> fdst (0 psi_R, 1 psi_I,
// 2 scratch), multiplier set `table`; the V term rides on the x pass.
template <typename T>
cudaError_t enqueue_apply(spstd_ctx *ctx, int fsrc, int fdst, int table, double bV, int reverse, cudaStream_t s,
                          LaunchTimer *timer = nullptr, int only_axis = -1)
{
    const spstd_config &cfg = ctx->cfg;
    const T *src = field_ptr<T>(ctx, fsrc);
    T *dst = field_ptr<T>(ctx, fdst);
    const T *mult = (const T *)ctx->ptr(ctx->L.mult) + (size_t)table * ctx->sum_n;
    const int64_t n0 = cfg.n[0], n1 = cfg.n[1], n2 = cfg.n[2];
    const int64_t *off = ctx->tab_off;
    int *status = (int *)ctx->ptr(ctx->L.status);
    int ax0 = 0;
    if constexpr (sizeof(T) == 4) {
        if (fused_active(ctx) && only_axis < 0 && fsrc <= 2 && fdst <= 2) {
            XyPassArgs xa{};
            xa.twx = (const float2 *)ctx->ptr(ctx->L.tw[0]);
            xa.twy = (const float2 *)ctx->ptr(ctx->L.tw[1]);
            xa.multx = (const float *)(mult + off[0]);
            xa.multy = (const float *)(mult + off[1]);
            xa.V = (const float *)ctx->ptr(ctx->L.V);
            xa.bV = (float)bV;
            xa.nx = (int)n0;
            xa.ny = (int)n1;
            xa.nz = (int)n2;
            xa.nyt = (int)(n0 / tma_cols_per_tile());
            xa.nxt = (int)(n1 / tma_rows_per_tile());
            unsigned *cnt = (unsigned *)ctx->ptr(ctx->L.xy);
            xa.claim = cnt;
            xa.ydone = cnt + 4;
            xa.xseen = cnt + 4 + n2;
            xa.status = status;
            SPSTD_TIMED(timer, s, 5,
                        launch_xypass_tma((int)n0, ctx->tmap[fsrc][0], ctx->tmap[fdst][0], ctx->tmap[fsrc][1],
                                          ctx->tmap[fdst][1], xa, s));
            ax0 = 2;
        } else if (fxy_active(ctx) && only_axis < 0 && fsrc <= 2 && fdst <= 2) {
            TmaPassArgs fa{};
            fa.tw = (const float2 *)ctx->ptr(ctx->L.tw[0]);
            fa.mult = (const float *)(mult + off[0]);
            fa.mult_y = (const float *)(mult + off[1]);
            fa.bV = (float)bV;
            fa.use_V = 1;
            fa.n_tiles = fxy_units(cfg.n);
            fa.status = status;
            fa.inject = status + 1;
            SPSTD_TIMED(timer, s, 5,
                        launch_pass_fxy((int)n0, ctx->fxmap[fsrc], ctx->fxmap[3], ctx->fxmap[fdst], fa, s));
            ax0 = 2;
        }
    }
    for (int ax = ax0; ax < cfg.dims; ++ax) {
        if (only_axis >= 0 && ax != only_axis) continue;
        const int rev = ax == 1 ? !reverse : reverse;
        const int64_t N = cfg.n[ax];
        const int sv = ctx->sched[ax];
        if (ax == 0 && ctx->long_x) {
            LongArgs<T> la{};
            la.src = src;
            la.dst = dst;
            la.V = (const T *)ctx->ptr(ctx->L.V);
            la.C = (cpx<T> *)ctx->ptr(ctx->L.lscr);
            la.tw1 = (const cpx<T> *)ctx->ptr(ctx->L.tw[0]);
            la.tw2 = la.tw1 + ctx->N1;
            la.twl = la.tw2 + ctx->N2;
            const double L = cfg.hi[0] - cfg.lo[0];
            la.scale = (T)(table_a(ctx, table) * (2.0 * kPi / L) * (2.0 * kPi / L) / (double)N);
            la.bV = (T)bV;
            la.nyquist_zero = cfg.nyquist_zero;
            la.N1 = ctx->N1;
            la.N2 = ctx->N2;
            la.n_rows = n1 * n2;
            la.n_pairs = (n1 * n2 + 1) / 2;
            for (int k = 0; k < 3; ++k) SPSTD_TIMED(timer, s, 0, launch_long_x<T>(la, s, k));
            continue;
        }
        if (ctx->dense[ax]) {
            DenseArgs<T> da{};
            da.src = src;
            da.dst = dst;
            da.V = (const T *)ctx->ptr(ctx->L.V);
            da.D = (const T *)ctx->ptr(ctx->L.dense[ax]);
            da.a = (T)table_scale(ctx, table);
            da.bV = (T)bV;
            da.use_V = ax == 0;
            da.n = (int)N;
            if (ax == 0) {
                da.stride = 1;
                da.inner = 1;
                da.outer_stride = n0;
                da.n_lines = n1 * n2;
            } else if (ax == 1) {
                da.stride = n0;
                da.inner = n0;
                da.outer_stride = n0 * n1;
                da.n_lines = n0 * n2;
            } else {
                da.stride = n0 * n1;
                da.inner = n0 * n1;
                da.outer_stride = 0;
                da.n_lines = n0 * n1;
            }
            if constexpr (sizeof(T) == 4) {
                // the tensor-core form (schedule 0 where it applies; 4 keeps the CUDA cores)
                if (dense_tc_axis(cfg, ax) && sv != 4) {
                    DenseTcArgs ta{};
                    ta.src = (const float *)src;
                    ta.dst = (float *)dst;
                    ta.V = (const float *)da.V;
                    ta.Dhi = (const float *)ctx->ptr(ctx->L.dense_tc[ax]);
                    ta.np = dense_tc_pad(N);
                    ta.Dlo = ta.Dhi + (size_t)ta.np * ta.np;
                    ta.a = (float)da.a;
                    ta.bV = (float)da.bV;
                    ta.use_V = da.use_V;
                    ta.n = (int)N;
                    ta.stride = da.stride;
                    ta.inner = da.inner;
                    ta.outer_stride = da.outer_stride;
                    ta.n_lines = da.n_lines;
                    ta.status = status;
                    SPSTD_TIMED(timer, s, ax, launch_dense_tc(ta, s));
                    continue;
                }
            }
            SPSTD_TIMED(timer, s, ax, Launch<T>::dense_pass(da, s));
            continue;
        }
        const cpx<T> *tw = (const cpx<T> *)ctx->ptr(ctx->L.tw[ax]);
        if constexpr (sizeof(T) == 4) {
            // reduce-add map of field f in the view of axis ax (null where none)
            auto redmap = [&](int f, int a) -> const CUtensorMap * {
                if (f <= 2) return a == 0 ? &ctx->xrmap[f] : &ctx->srmap[f][a - 1];
                if (f <= 6 && ctx->rk_tma[a]) return &ctx->rkmap[f - 3][a];
                return nullptr;
            };
            const bool std_fields = fsrc <= 2 && fdst <= 2;
            // the RK4 stage fields have block-tile reduce-add maps only
            const bool red = ctx->tma[ax] && (sv == 0 || (sv == 6 && !std_fields)) && redmap(fsrc, ax) &&
                             redmap(fdst, ax);
            const bool st = ctx->tma_st[ax] && sv == 5 && std_fields;
            const bool xw = ax == 0 && ctx->xw_ok && sv == 6 && std_fields;
            if (red || st || xw) {
                TmaPassArgs ta{};
                ta.tw = (const float2 *)tw;
                ta.mult = (const float *)(mult + off[ax]);
                ta.V = (const float *)ctx->ptr(ctx->L.V);
                ta.bV = (float)bV;
                ta.use_V = ax == 0;
                ta.rows = (int)(n1 * n2);
                ta.axis = ax;
                ta.reverse = rev;
                ta.status = status;
                ta.nx = (int)n0;
                ta.planes = red_planes(cfg.n, ax);
                ta.inject = status + 1;
                if (ax == 0 && (red || xw) && ta.use_V && ctx->vsep) {
                    ta.vx = (const float *)ctx->ptr(ctx->L.vsep_x);
                    ta.vyz = (const float *)ctx->ptr(ctx->L.vsep_yz);
                }
                if (xw) {
                    const int R = xwarp_rows((int)N);
                    ta.n_tiles = (int)((n1 * n2 + R - 1) / R);
                    SPSTD_TIMED(timer, s, 0,
                                launch_pass_xwarp((int)N, ctx->xwmap[fsrc], ctx->xwmap[3], ctx->xwmap[fdst], ta, s));
                } else if (red) {
                    ta.n_tiles = tmared_tiles(ax, cfg.n, &ta.n_xt);
                    SPSTD_TIMED(timer, s, ax,
                                launch_pass_tmared(ax, (int)N, *redmap(fsrc, ax), ctx->xrmap[3], *redmap(fdst, ax), ta,
                                                   s));
                } else {
                    if (ax == 0) {
                        ta.n_tiles = (int)((n1 * n2 + tma_rows_per_tile() - 1) / tma_rows_per_tile());
                    } else {
                        ta.n_xt = (int)((n0 + tma_cols_per_tile() - 1) / tma_cols_per_tile());
                        ta.n_tiles = ta.n_xt * (int)(ax == 1 ? n2 : n1);
                    }
                    SPSTD_TIMED(timer, s, ax,
                                launch_pass_tma(ax, (int)N, ctx->tmap[fsrc][ax], ctx->tmap[fdst][ax], ta, s));
                }
                continue;
            }
        }
        PassArgs<T> a{};
        a.src = src;
        a.dst = dst;
        a.tw = tw;
        a.mult = mult + off[ax];
        a.reverse = rev;
        if (ax == 0) {
            a.V = (const T *)ctx->ptr(ctx->L.V);
            a.bV = (T)bV;
            a.use_V = 1;
            a.n_rows = n1 * n2;
            SPSTD_TIMED(timer, s, 0,
                        (sv >= 1 && sv <= 3) ? xpass_sched<T>((int)N, sv, a, s) : Launch<T>::xpass((int)N, a, s));
        } else {
            a.stride = ax == 1 ? n0 : n0 * n1;
            a.outer_stride = ax == 1 ? n0 * n1 : n0;
            a.n_outer = ax == 1 ? n2 : n1;
            a.nx = (int)n0;
            SPSTD_TIMED(timer, s, ax,
                        (sv >= 1 && sv <= 3) ? spass_sched<T>((int)N, sv, a, s) : Launch<T>::spass((int)N, a, s));
        }
    }
    return cudaSuccess;
}

template <typename T>
ProbeArgs probe_args(spstd_ctx *ctx)
{
    ProbeArgs p{};
    p.n_probe = ctx->cfg.n_probe;
    for (int q = 0; q < p.n_probe; ++q) p.idx[q] = ctx->cfg.probe_idx[q];
    p.ring = (double2 *)ctx->ptr(ctx->L.ring);
    p.cap = ctx->cfg.probe_capacity;
    p.counter = (int64_t *)ctx->ptr(ctx->L.counter);
    return p;
}

// nsteps full steps of Eq. 17/18 (2D/3D): every half-stage as x, y(, z)
// passes, then the probe recorder.  With ctx->merge, the last half-stage of
// each step but the final one is fused with the first of the next step (same
// field, summed coefficient), and the probe between them is interpolated
// exactly from a snapshot taken before the fused half-stage.
template <typename T>
cudaError_t enqueue_steps(spstd_ctx *ctx, int64_t nsteps, cudaStream_t s, LaunchTimer *timer = nullptr)
{
    T *psi[2] = {(T *)ctx->ptr(ctx->L.psi[0]), (T *)ctx->ptr(ctx->L.psi[1])};
    const bool probes = ctx->cfg.n_probe > 0;
    double2 *snap = (double2 *)ctx->ptr(ctx->L.snap);
    const int nh = (int)ctx->hs.size();
    int parity = 0;
    for (int64_t i = 0; i < nsteps; ++i) {
        const bool fused_in = ctx->merge && i > 0;            // first half-stage already applied
        const bool fused_out = ctx->merge && i + 1 < nsteps;  // last half-stage fused with the next
        for (int k = fused_in ? 1 : 0; k < nh; ++k) {
            if (k == nh - 1 && fused_out) {
                const HalfStage &h = ctx->merged;
                if (probes)
                    SPSTD_TIMED(timer, s, 3, Launch<T>::probe_snapshot(psi[0], psi[1], probe_args<T>(ctx), snap, s));
                cudaError_t e = enqueue_apply<T>(ctx, 1 - h.dst, h.dst, h.table, h.bV, parity, s, timer);
                if (e != cudaSuccess) return e;
                parity ^= 1;
                if (probes)
                    SPSTD_TIMED(timer, s, 3,
                                Launch<T>::probe_merged(psi[0], psi[1], probe_args<T>(ctx), snap, ctx->merge_alpha,
                                                        h.dst, s));
            } else {
                const HalfStage &h = ctx->hs[k];
                cudaError_t e = enqueue_apply<T>(ctx, 1 - h.dst, h.dst, h.table, h.bV, parity, s, timer);
                if (e != cudaSuccess) return e;
                parity ^= 1;
            }
        }
        if (probes && !fused_out)
            SPSTD_TIMED(timer, s, 3, Launch<T>::probe(psi[0], psi[1], probe_args<T>(ctx), s));
    }
    return cudaSuccess;
}

// With merged boundaries a call of n steps is: the first half-stage, n - 1
// units, the tail.  A unit is the inner half-stages of a step followed by the
// fused boundary (its last half-stage + the next step's first) and the
// interpolated probe; the tail is the inner half-stages, the last half-stage
// and the probe.  Units are what the captured graph replays.
template <typename T>
cudaError_t enqueue_merged_piece(spstd_ctx *ctx, int piece, int64_t units, cudaStream_t s,
                                 LaunchTimer *timer = nullptr)
{
    T *psi[2] = {(T *)ctx->ptr(ctx->L.psi[0]), (T *)ctx->ptr(ctx->L.psi[1])};
    const bool probes = ctx->cfg.n_probe > 0;
    double2 *snap = (double2 *)ctx->ptr(ctx->L.snap);
    const int nh = (int)ctx->hs.size();
    int parity = 0;
    auto apply = [&](const HalfStage &h) {
        cudaError_t e = enqueue_apply<T>(ctx, 1 - h.dst, h.dst, h.table, h.bV, parity, s, timer);
        parity ^= 1;
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (piece == 0) return apply(ctx->hs[0]);  // head
    if (piece == 1) {                          // units
        for (int64_t u = 0; u < units; ++u) {
            for (int k = 1; k < nh - 1; ++k)
                if ((e = apply(ctx->hs[k])) != cudaSuccess) return e;
            if (probes)
                SPSTD_TIMED(timer, s, 3, Launch<T>::probe_snapshot(psi[0], psi[1], probe_args<T>(ctx), snap, s));
            if ((e = apply(ctx->merged)) != cudaSuccess) return e;
            if (probes)
                SPSTD_TIMED(timer, s, 3,
                            Launch<T>::probe_merged(psi[0], psi[1], probe_args<T>(ctx), snap, ctx->merge_alpha,
                                                    ctx->merged.dst, s));
        }
        return cudaSuccess;
    }
    for (int k = 1; k < nh; ++k)  // tail
        if ((e = apply(ctx->hs[k])) != cudaSuccess) return e;
    if (probes) SPSTD_TIMED(timer, s, 3, Launch<T>::probe(psi[0], psi[1], probe_args<T>(ctx), s));
    return cudaSuccess;
}

// Kernel launches enqueue_steps(n) issues.
// Kernel launches of one H-apply between the state fields: one per axis, three
// for a four-step x axis, one for a fused x-y pair.
inline int64_t apply_launches(const spstd_ctx *ctx)
{
    return ctx->cfg.dims + (ctx->long_x ? 2 : 0) - (fused_active(ctx) || fxy_active(ctx) ? 1 : 0);
}

// A 1D grid runs all steps of a call in one resident launch unless its line
// is too long for one block.
inline bool resident_path(const spstd_ctx *ctx) { return ctx->cfg.dims == 1 && !ctx->long_x; }

inline int64_t launches_for_steps(const spstd_ctx *ctx, int64_t n)
{
    if (n <= 0) return 0;
    const int64_t nh = (int64_t)ctx->hs.size();
    const int64_t halfstages = ctx->merge ? n * nh - (n - 1) : n * nh;
    // a merged boundary records its probe with a snapshot and an interpolating recorder
    const int64_t probe = ctx->cfg.n_probe > 0 ? (ctx->merge ? 2 * n - 1 : n) : 0;
    return halfstages * apply_launches(ctx) + probe;
}

template <typename T>
cudaError_t launch_dense_resident(spstd_ctx *ctx, int64_t nsteps, LaunchTimer *timer)
{
    DenseResidentArgs<T> r{};
    r.psiR = field_ptr<T>(ctx, 0);
    r.psiI = field_ptr<T>(ctx, 1);
    r.V = (const T *)ctx->ptr(ctx->L.V);
    r.D = (const T *)ctx->ptr(ctx->L.dense[0]);
    r.nh = (int)ctx->hs.size();
    for (int h = 0; h < r.nh; ++h) {
        r.a[h] = (T)ctx->hs[h].scale;
        r.bV[h] = (T)ctx->hs[h].bV;
        r.hfield[h] = ctx->hs[h].dst;
    }
    r.n = (int)ctx->cfg.n[0];
    r.nsteps = nsteps;
    ProbeArgs p = probe_args<T>(ctx);
    r.n_probe = p.n_probe;
    for (int q = 0; q < p.n_probe; ++q) r.probe_idx[q] = p.idx[q];
    r.ring = p.ring;
    r.cap = p.cap;
    r.counter = p.counter;
    SPSTD_TIMED(timer, ctx->stream, 4, Launch<T>::dense_resident1d(r, ctx->stream));
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_resident(spstd_ctx *ctx, int64_t nsteps, LaunchTimer *timer)
{
    const spstd_config &cfg = ctx->cfg;
    if (ctx->dense[0]) return launch_dense_resident<T>(ctx, nsteps, timer);
    ResidentArgs<T> r{};
    r.psiR = (T *)ctx->ptr(ctx->L.psi[0]);
    r.psiI = (T *)ctx->ptr(ctx->L.psi[1]);
    r.V = (const T *)ctx->ptr(ctx->L.V);
    r.tw = (const cpx<T> *)ctx->ptr(ctx->L.tw[0]);
    r.mult = (const T *)ctx->ptr(ctx->L.mult);
    r.nh = (int)ctx->hs.size();
    for (int h = 0; h < r.nh; ++h) {
        r.bV[h] = (T)ctx->hs[h].bV;
        r.hfield[h] = ctx->hs[h].dst;
        r.htable[h] = ctx->hs[h].table;
    }
    r.nsteps = nsteps;
    ProbeArgs p = probe_args<T>(ctx);
    r.n_probe = p.n_probe;
    for (int q = 0; q < p.n_probe; ++q) r.probe_idx[q] = p.idx[q];
    r.ring = p.ring;
    r.cap = p.cap;
    r.counter = p.counter;
    SPSTD_TIMED(timer, ctx->stream, 4, Launch<T>::resident1d((int)cfg.n[0], r, ctx->stream));
    return cudaSuccess;
}

// Raises the shared-memory limits of the pass kernels once, outside any capture.
template <typename T>
spstd_status prepare_kernels(spstd_ctx *ctx)
{
    const spstd_config &cfg = ctx->cfg;
    PassArgs<T> none{};
    if (ctx->long_x) SPSTD_CU(ctx, prepare_long_x<T>(ctx->N1, ctx->N2));
    else if (!ctx->dense[0]) SPSTD_CU(ctx, Launch<T>::xpass((int)cfg.n[0], none, ctx->stream));
    none.nx = (int)cfg.n[0];
    if (cfg.dims > 1 && !ctx->dense[1]) SPSTD_CU(ctx, Launch<T>::spass((int)cfg.n[1], none, ctx->stream));
    if (cfg.dims == 3 && !ctx->dense[2]) SPSTD_CU(ctx, Launch<T>::spass((int)cfg.n[2], none, ctx->stream));
    if (ctx->fuse_xy) SPSTD_CU(ctx, prepare_xypass_tma((int)cfg.n[0]));
    for (int ax = 0; ax < cfg.dims; ++ax) {
        if (dense_tc_axis(cfg, ax)) SPSTD_CU(ctx, launch_dense_tc(DenseTcArgs{}, ctx->stream));
        if (ctx->tma[ax]) SPSTD_CU(ctx, prepare_pass_tmared(ax, (int)cfg.n[ax], cfg.n[0], red_planes(cfg.n, ax)));
        if (ctx->tma_st[ax]) SPSTD_CU(ctx, prepare_pass_tma(ax, (int)cfg.n[ax]));
        if (ax == 0 && ctx->xw_ok && ctx->sched[0] == 6) SPSTD_CU(ctx, prepare_pass_xwarp((int)cfg.n[0]));
        if (ax == 0 && ctx->fxy_ok) SPSTD_CU(ctx, prepare_pass_fxy((int)cfg.n[0], false));
        const int sv = ctx->sched[ax];
        if (sv >= 1 && sv <= 3) {
            PassArgs<T> z{};
            SPSTD_CU(ctx, ax == 0 ? xpass_sched<T>((int)cfg.n[ax], sv, z, ctx->stream)
                                  : spass_sched<T>((int)cfg.n[ax], sv, z, ctx->stream));
        }
    }
    return SPSTD_OK;
}

// One classical Runge-Kutta step (the comparison scheme of Fig. 3): four
// stages, each H applied to the stage state's two fields by the pass kernels,
// then the stage update; the state becomes the accumulated sum; then probes.
template <typename T>
cudaError_t enqueue_rk4_step(spstd_ctx *ctx, cudaStream_t s, LaunchTimer *timer = nullptr)
{
    const size_t bytes = sizeof(T) * ctx->ntot;
    T *y[2] = {field_ptr<T>(ctx, 0), field_ptr<T>(ctx, 1)};
    T *t[2] = {field_ptr<T>(ctx, 3), field_ptr<T>(ctx, 4)};
    T *h[2] = {field_ptr<T>(ctx, 5), field_ptr<T>(ctx, 6)};
    T *acc[2] = {field_ptr<T>(ctx, 7), field_ptr<T>(ctx, 8)};
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double a[4] = {0.0, 0.5, 0.5, 1.0};
    const double k = ctx->dt / ctx->cfg.hbar;
    const int tH = 2 * ctx->m;
    cudaError_t e;
    for (int j = 0; j < 4; ++j) {
        for (int f = 0; f < 2; ++f)
            if ((e = cudaMemsetAsync(h[f], 0, bytes, s)) != cudaSuccess) return e;
        // the first stage's state is y itself (fields 0, 1); later ones t (3, 4)
        const int tR = j == 0 ? 0 : 3, tI = j == 0 ? 1 : 4;
        if ((e = enqueue_apply<T>(ctx, tI, 5, tH, 1.0, 0, s, timer)) != cudaSuccess) return e;  // h_R = H t_I
        if ((e = enqueue_apply<T>(ctx, tR, 6, tH, 1.0, 1, s, timer)) != cudaSuccess) return e;  // h_I = H t_R
        // the running sum starts from y and, at the last stage, lands in y
        const T *aR = j == 0 ? y[0] : acc[0], *aI = j == 0 ? y[1] : acc[1];
        T *oR = j == 3 ? y[0] : acc[0], *oI = j == 3 ? y[1] : acc[1];
        e = Launch<T>::rk4_update(y[0], y[1], h[0], h[1], aR, aI, oR, oI, t[0], t[1], ctx->ntot, (T)(b[j] * k),
                                  (T)(j < 3 ? a[j + 1] * k : 0.0), j == 3, s);
        if (e != cudaSuccess) return e;
    }
    if (ctx->cfg.n_probe > 0) SPSTD_TIMED(timer, s, 3, Launch<T>::probe(y[0], y[1], probe_args<T>(ctx), s));
    return cudaSuccess;
}

// A step followed by the eigenstate accumulation (every step ends at a full state).
template <typename T>
cudaError_t enqueue_eigen_step(spstd_ctx *ctx, cudaStream_t s, LaunchTimer *timer = nullptr)
{
    cudaError_t e = ctx->rk4 ? enqueue_rk4_step<T>(ctx, s, timer) : enqueue_steps<T>(ctx, 1, s, timer);
    if (e != cudaSuccess) return e;
    int64_t *step = (int64_t *)ctx->ptr(ctx->L.eig_step);
    SPSTD_TIMED(timer, s, 3,
                Launch<T>::eigen_accum(field_ptr<T>(ctx, 0), field_ptr<T>(ctx, 1), (double2 *)ctx->ptr(ctx->L.eig_acc),
                                       ctx->ntot, ctx->eig_n, (const double *)ctx->ptr(ctx->L.eig_theta),
                                       ctx->eig_window, step, (unsigned *)(step + 1), s));
    return cudaSuccess;
}

// Captures the graph that 2D/3D steps replay: kGraphSteps units with merged
// step boundaries, else kGraphSteps steps.  It is done on the first step call
// of a context (or the first after a change that dropped the graph), whatever
// that call's length, so that the capture and instantiation never fall inside
// a later, longer call.
template <typename T>
spstd_status ensure_graph(spstd_ctx *ctx)
{
    if (ctx->gexec || ctx->cfg.no_graph) return SPSTD_OK;
    spstd_status ps = prepare_kernels<T>(ctx);
    if (ps != SPSTD_OK) return ps;
    cudaGraph_t g = nullptr;
    SPSTD_CU(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = ctx->merge ? enqueue_merged_piece<T>(ctx, 1, kGraphSteps, ctx->cap_stream)
                               : enqueue_steps<T>(ctx, kGraphSteps, ctx->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e != cudaSuccess ? e : e2, "graph capture");
    }
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->gexec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    return SPSTD_OK;
}

template <typename T>
spstd_status step_impl(spstd_ctx *ctx, int64_t nsteps)
{
    if (ctx->rk4 && !ctx->eig_active) {
        for (int64_t i = 0; i < nsteps; ++i) SPSTD_CU(ctx, enqueue_rk4_step<T>(ctx, ctx->stream));
        ctx->steps_taken += nsteps;
        return SPSTD_OK;
    }
    if (ctx->eig_active) {
        for (int64_t i = 0; i < nsteps; ++i) SPSTD_CU(ctx, enqueue_eigen_step<T>(ctx, ctx->stream));
        ctx->steps_taken += nsteps;
        return SPSTD_OK;
    }
    if (resident_path(ctx)) {
        SPSTD_CU(ctx, launch_resident<T>(ctx, nsteps, nullptr));
        ctx->steps_taken += nsteps;
        return SPSTD_OK;
    }
    spstd_status gs = ensure_graph<T>(ctx);
    if (gs != SPSTD_OK) return gs;
    cudaError_t e;
    if (ctx->merge) {
        // head, graph-replayed units, remaining units, tail
        const int64_t units = nsteps - 1;
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 0, 0, ctx->stream));
        int64_t done = 0;
        if (ctx->gexec) {
            for (int64_t r = 0; r < units / kGraphSteps; ++r) SPSTD_CU(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream));
            done = units / kGraphSteps * kGraphSteps;
        }
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 1, units - done, ctx->stream));
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 2, 0, ctx->stream));
        ctx->steps_taken += nsteps;
        return SPSTD_OK;
    }
    if (ctx->gexec) {
        const int64_t reps = nsteps / kGraphSteps;
        for (int64_t i = 0; i < reps; ++i) SPSTD_CU(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream));
        nsteps -= reps * kGraphSteps;
        ctx->steps_taken += reps * kGraphSteps;
    }
    if (nsteps > 0) {
        e = enqueue_steps<T>(ctx, nsteps, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
        ctx->steps_taken += nsteps;
    }
    return SPSTD_OK;
}

}  // namespace spstd_host
