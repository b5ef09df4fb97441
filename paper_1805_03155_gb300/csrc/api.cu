// api.cu -- the C ABI of include/spstd.h: validation, device workspace
// layout, FP64 host tables, the time-step driver (direct launches and captured
// CUDA graphs) and the host halves of the reductions and the spectrum.
//
// The host code here computes only setup quantities (coefficient presets,
// the stability limit of Eq. 23-25, twiddle and k^2 tables, dispersion
// inversion of a few spectrum peaks); every step of the time integration,
// every reduction and every spectrum runs in the CUDA kernels.
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

#include "../../include/spstd.h"
#include "../../include/spstd_testing.h"
#include "launch.cuh"
#include "longline.h"
#include "pass_tma_launch.h"
#include "pass_xy.cuh"
#include "sched.h"
#include "spectrum.h"

using namespace spstd;

namespace {

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

struct Layout {
    size_t psi[2], V, vsep_x, vsep_yz, tmp, staging, ring, counter, status, snap, partial, dout, tw[3], mult, dense[3], spec;
    size_t eig_acc, eig_theta, eig_step, rk[6], lscr, xy, total;
};

// Periodic lengths 3 * 2^k that the 2D/3D pass kernels transform with a
// radix-3 first stage (line_e and the plans of fft_line.cuh).
bool is_radix3_len(int64_t n) { return n == 24 || n == 48 || n == 96 || n == 192 || n == 384; }

// An axis uses the FFT passes when it is periodic with a power-of-two length
// within the FFT limits, or (2D/3D grids) one of the radix-3 lengths;
// otherwise the dense operator (n <= SPSTD_MAX_DENSE_N).
bool axis_is_fft(const spstd_config &cfg, int a)
{
    const int64_t n = cfg.n[a];
    if (cfg.bc[a] != SPSTD_PERIODIC) return false;
    if ((n & (n - 1)) != 0) return cfg.dims > 1 && is_radix3_len(n);
    const int64_t lim = cfg.dims == 1 ? (cfg.precision == 32 ? 8192 : 4096) : 1024;
    return n >= 2 && n <= lim;
}

// The x axis of a periodic power-of-two length beyond the on-chip limit runs
// the four-step pass (up to 2^22 points).
bool axis_is_long(const spstd_config &cfg, int a)
{
    const int64_t n = cfg.n[a];
    return a == 0 && cfg.bc[a] == SPSTD_PERIODIC && (n & (n - 1)) == 0 && !axis_is_fft(cfg, a) && n <= kMaxLongN;
}

// 3D FP32 grids whose x and y axes both take the pipelined passes at the same
// length can run them as one fused launch (pass_xy.cuh).
bool xy_fusable(const spstd_config &cfg)
{
    auto tma_len = [](int64_t n) { return n == 64 || n == 128 || n == 256; };
    return cfg.precision == 32 && cfg.dims == 3 && cfg.n[0] == cfg.n[1] && tma_len(cfg.n[0]) &&
           cfg.bc[0] == SPSTD_PERIODIC && cfg.bc[1] == SPSTD_PERIODIC && cfg.n[2] >= 2;
}

// Entries of an axis in each multiplier row (the four-step pass computes its
// multipliers from the wrapped index instead).
int64_t table_len(const spstd_config &cfg, int a) { return a < cfg.dims && !axis_is_long(cfg, a) ? cfg.n[a] : 0; }

// Points per cell length: periodic L/n, Dirichlet L/(n+1), Neumann L/(n-1).
double axis_spacing(const spstd_config &cfg, int a)
{
    const double L = cfg.hi[a] - cfg.lo[a];
    const int64_t n = cfg.n[a];
    return cfg.bc[a] == SPSTD_DIRICHLET ? L / (double)(n + 1) : cfg.bc[a] == SPSTD_NEUMANN ? L / (double)(n - 1)
                                                                                           : L / (double)n;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int64_t next_pow2(int64_t v)
{
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// ---- integrator coefficients (Eq. 17) ---------------------------------------
bool preset_coefficients(int id, int *m, double *c, double *d)
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
double step_trace(int m, const double *c, const double *d, double s)
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

double stability_s_star(int m, const double *c, const double *d)
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
double scheme_s_star(int preset, int m, const double *c, const double *d)
{
    if (preset == SPSTD_RK4) return 2.0 * std::sqrt(2.0);
    return stability_s_star(m, c, d);
}

// Phase advance per step of the mode with w dt = s. m = 0 is the classical
// Runge-Kutta scheme: its factor R(-is) = 1 - is - s^2/2 + is^3/6 + s^4/24 is
// not unimodular; the angle of exp(-i theta) is -arg R, taken in [0, pi].
double map_angle(int m, const double *c, const double *d, double s)
{
    if (m == 0) return std::fabs(std::atan2(s - s * s * s / 6.0, 1.0 - 0.5 * s * s + s * s * s * s / 24.0));
    double t = 0.5 * step_trace(m, c, d, s);
    t = std::min(1.0, std::max(-1.0, t));
    return std::acos(t);
}

// s with map_angle(s) = theta on the first increasing branch (Eq. 24/25: the
// eigenvalues of a det-1 map are exp(+-i theta), theta = arccos(tr/2)).
double dispersion_inverse(int m, const double *c, const double *d, double s_star, double theta)
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

double w_max_of(const spstd_config &cfg, double vmax)
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
spstd_status validate(const spstd_config *cfg, std::string *why, int *m, double *c, double *d)
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

int64_t effective_max_nfft(const spstd_config &cfg)
{
    if (cfg.max_nfft > 0) return cfg.max_nfft;
    return std::max<int64_t>(4, next_pow2(4 * cfg.probe_capacity));
}

int64_t vsep_rows_padded(int64_t rows) { return (rows + 127) / 128 * 128; }

Layout make_layout(const spstd_config &cfg, int m)
{
    Layout L{};
    const int64_t ntot = cfg.n[0] * cfg.n[1] * cfg.n[2];
    const size_t es = cfg.precision == 32 ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes);
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

}  // namespace

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
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    // pipelined FP32 passes: tensor maps [field: psi_R, psi_I, tmp][view: x, y, z]
    // default (reduce-add) passes: tma[axis]; x view of psi_R, psi_I, tmp, V;
    // y and z views of the fields, with the boxes of pass_tmared.cuh
    bool tma[3] = {false, false, false};
    CUtensorMap xrmap[4];
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

namespace {

spstd_status fail(spstd_ctx *ctx, spstd_status s, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return s;
}
spstd_status cuda_fail(spstd_ctx *ctx, cudaError_t e, const char *where)
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
spstd_status check_device_status(spstd_ctx *ctx)
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

void drop_graph(spstd_ctx *ctx)
{
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
}

// k^2 of DFT index j on an n-point axis of period L (wrapped index, Eq. 8).
double k2_of(int64_t j, int64_t n, double L, int nyquist_zero)
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
std::vector<double> dense_operator(const spstd_config &cfg, int axis)
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
double table_a(const spstd_ctx *ctx, int t)
{
    const spstd_config &cfg = ctx->cfg;
    const int m = ctx->m;
    if (t == 2 * m + 1) return ctx->merge ? ctx->merged.a : 0.0;
    if (t == 2 * m) return cfg.hbar * cfg.hbar / (2.0 * cfg.mass);
    return (t & 1) ? -ctx->d[t / 2] * ctx->dt * cfg.hbar / (2.0 * cfg.mass)
                   : +ctx->c[t / 2] * ctx->dt * cfg.hbar / (2.0 * cfg.mass);
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
    }
    // the host vectors die here: wait until the copies have read them
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return SPSTD_OK;
}

// cuTensorMapEncodeTiled from the driver, without linking libcuda.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
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
bool encode_map(CUtensorMap *m, void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
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
int red_planes(const int64_t *n, int ax)
{
    if (ax == 0) return 1;
    return tmared_planes((int)n[ax], tmared_pairs((int)n[ax], n[0]), ax == 1 ? n[2] : n[1]);
}

// 4D FP32 tensor map (dims d[0] fastest; strides of dims 1..3 in elements)
// with the given box; out-of-range box elements load as zero and are not
// written back.
bool encode_map4(CUtensorMap *m, void *base, const uint64_t *d, const uint64_t *stride, const uint32_t *box)
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
bool encode_red_map(CUtensorMap *m, void *base, const int64_t *n, int v)
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
void setup_tma(spstd_ctx *ctx)
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

spstd_status set_dt(spstd_ctx *ctx, double vmax)
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
double table_scale(const spstd_ctx *ctx, int table)
{
    if (table == 2 * ctx->m + 1) return ctx->merged.scale;
    if (table >= 2 * ctx->m) return ctx->cfg.hbar;
    const int l = table / 2;
    return (table & 1) ? -ctx->d[l] * ctx->dt : ctx->c[l] * ctx->dt;
}

// Whether an H-apply between psi_R, psi_I and the scratch field runs x and y as one launch.
bool fused_active(const spstd_ctx *ctx) { return ctx->fuse_xy && ctx->sched[0] == 0 && ctx->sched[1] == 0; }

// Whether H-applies between the state fields run x and y as the fused reduce-add pass.
bool fxy_active(const spstd_ctx *ctx)
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
            SPSTD_TIMED(timer, s, ax, Launch<T>::dense_pass(da, s));
            continue;
        }
        const cpx<T> *tw = (const cpx<T> *)ctx->ptr(ctx->L.tw[ax]);
        if constexpr (sizeof(T) == 4) {
            const bool red = ctx->tma[ax] && sv == 0, st = ctx->tma_st[ax] && sv == 5;
            if ((red || st) && fsrc <= 2 && fdst <= 2) {
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
                if (ax == 0 && red && ta.use_V && ctx->vsep) {
                    ta.vx = (const float *)ctx->ptr(ctx->L.vsep_x);
                    ta.vyz = (const float *)ctx->ptr(ctx->L.vsep_yz);
                }
                if (red) {
                    ta.n_tiles = tmared_tiles(ax, cfg.n, &ta.n_xt);
                    if (ax == 0)
                        SPSTD_TIMED(timer, s, ax,
                                    launch_pass_tmared(0, (int)N, ctx->xrmap[fsrc], ctx->xrmap[3], ctx->xrmap[fdst],
                                                       ta, s));
                    else
                        SPSTD_TIMED(timer, s, ax,
                                    launch_pass_tmared(ax, (int)N, ctx->srmap[fsrc][ax - 1], ctx->xrmap[3],
                                                       ctx->srmap[fdst][ax - 1], ta, s));
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
int64_t apply_launches(const spstd_ctx *ctx)
{
    return ctx->cfg.dims + (ctx->long_x ? 2 : 0) - (fused_active(ctx) || fxy_active(ctx) ? 1 : 0);
}

// A 1D grid runs all steps of a call in one resident launch unless its line
// is too long for one block.
bool resident_path(const spstd_ctx *ctx) { return ctx->cfg.dims == 1 && !ctx->long_x; }

int64_t launches_for_steps(const spstd_ctx *ctx, int64_t n)
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
        if (ctx->tma[ax]) SPSTD_CU(ctx, prepare_pass_tmared(ax, (int)cfg.n[ax], cfg.n[0], red_planes(cfg.n, ax)));
        if (ctx->tma_st[ax]) SPSTD_CU(ctx, prepare_pass_tma(ax, (int)cfg.n[ax]));
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
    cudaError_t e;
    for (int f = 0; f < 2; ++f) {
        if ((e = cudaMemcpyAsync(t[f], y[f], bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(acc[f], y[f], bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    }
    const int tH = 2 * ctx->m;
    for (int j = 0; j < 4; ++j) {
        for (int f = 0; f < 2; ++f)
            if ((e = cudaMemsetAsync(h[f], 0, bytes, s)) != cudaSuccess) return e;
        if ((e = enqueue_apply<T>(ctx, 4, 5, tH, 1.0, 0, s, timer)) != cudaSuccess) return e;  // h_R = H t_I
        if ((e = enqueue_apply<T>(ctx, 3, 6, tH, 1.0, 1, s, timer)) != cudaSuccess) return e;  // h_I = H t_R
        e = Launch<T>::rk4_update(y[0], y[1], h[0], h[1], acc[0], acc[1], t[0], t[1], ctx->ntot, (T)(b[j] * k),
                                  (T)(j < 3 ? a[j + 1] * k : 0.0), j == 3, s);
        if (e != cudaSuccess) return e;
    }
    for (int f = 0; f < 2; ++f)
        if ((e = cudaMemcpyAsync(y[f], acc[f], bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
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

template <typename T>
spstd_status step_impl(spstd_ctx *ctx, int64_t nsteps)
{
    T *psi0 = (T *)ctx->ptr(ctx->L.psi[0]);
    T *psi1 = (T *)ctx->ptr(ctx->L.psi[1]);
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
    cudaError_t e;
    if (ctx->merge) {
        // head, graph-replayed units, remaining units, tail
        const int64_t units = nsteps - 1;
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 0, 0, ctx->stream));
        int64_t done = 0;
        if (units >= kGraphSteps && !ctx->cfg.no_graph) {
            if (!ctx->gexec) {
                spstd_status ps = prepare_kernels<T>(ctx);
                if (ps != SPSTD_OK) return ps;
                cudaGraph_t g = nullptr;
                SPSTD_CU(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
                e = enqueue_merged_piece<T>(ctx, 1, kGraphSteps, ctx->cap_stream);
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
            }
            for (int64_t r = 0; r < units / kGraphSteps; ++r) SPSTD_CU(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream));
            done = units / kGraphSteps * kGraphSteps;
        }
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 1, units - done, ctx->stream));
        SPSTD_CU(ctx, enqueue_merged_piece<T>(ctx, 2, 0, ctx->stream));
        ctx->steps_taken += nsteps;
        return SPSTD_OK;
    }
    if (nsteps >= kGraphSteps && !ctx->cfg.no_graph) {
        if (!ctx->gexec) {
            spstd_status ps = prepare_kernels<T>(ctx);
            if (ps != SPSTD_OK) return ps;
            cudaGraph_t g = nullptr;
            SPSTD_CU(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            e = enqueue_steps<T>(ctx, kGraphSteps, ctx->cap_stream);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(ctx->cap_stream, &g);
                if (g) cudaGraphDestroy(g);
                return cuda_fail(ctx, e, "graph capture");
            }
            SPSTD_CU(ctx, cudaStreamEndCapture(ctx->cap_stream, &g));
            e = cudaGraphInstantiate(&ctx->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->gexec = nullptr;
                return cuda_fail(ctx, e, "cudaGraphInstantiate");
            }
        }
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

}  // namespace

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
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_status(ctx);
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
    // kernel arguments name the tables (or not): replayed graphs are rebuilt
    drop_graph(ctx);
    ctx->vsep = false;
    // the table form of the x pass exists for power-of-two lines
    if (ctx->cfg.precision == 32 && ctx->tma[0] && is_pow2(ctx->cfg.n[0])) {
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
    spstd_status s = ctx->cfg.precision == 32 ? upload_field<float>(ctx, psiR, ctx->L.psi[0])
                                              : upload_field<double>(ctx, psiR, ctx->L.psi[0]);
    if (s != SPSTD_OK) return s;
    s = ctx->cfg.precision == 32 ? upload_field<float>(ctx, psiI, ctx->L.psi[1])
                                 : upload_field<double>(ctx, psiI, ctx->L.psi[1]);
    if (s != SPSTD_OK) return s;
    SPSTD_CU(ctx, cudaMemsetAsync(ctx->ptr(ctx->L.counter), 0, 8, ctx->stream));
    ctx->steps_taken = 0;
    // N0 = dV sum(psi_R^2 + psi_I^2) of the given state, for the divergence rule
    double acc = 0.0, dV = 1.0;
    for (int64_t i = 0; i < ctx->ntot; ++i) acc += psiR[i] * psiR[i] + psiI[i] * psiI[i];
    for (int a = 0; a < ctx->cfg.dims; ++a) dV *= axis_spacing(ctx->cfg, a);
    ctx->norm0 = dV * acc;
    return SPSTD_OK;
}

spstd_status spstd_get_state(spstd_ctx *ctx, double *psiR, double *psiI)
{
    if (!ctx || !psiR || !psiI) return SPSTD_EINVAL;
    spstd_status s = ctx->cfg.precision == 32 ? download_field<float>(ctx, ctx->ptr(ctx->L.psi[0]), psiR)
                                              : download_field<double>(ctx, ctx->ptr(ctx->L.psi[0]), psiR);
    if (s != SPSTD_OK) return s;
    return ctx->cfg.precision == 32 ? download_field<float>(ctx, ctx->ptr(ctx->L.psi[1]), psiI)
                                    : download_field<double>(ctx, ctx->ptr(ctx->L.psi[1]), psiI);
}

spstd_status spstd_step(spstd_ctx *ctx, int64_t nsteps)
{
    if (!ctx || nsteps < 0) return SPSTD_EINVAL;
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
    std::vector<double2> row(C);
    SPSTD_CU(ctx, cudaMemcpyAsync(row.data(), (double2 *)ctx->ptr(ctx->L.ring) + (size_t)p * C, sizeof(double2) * C,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPSTD_CU(ctx, cudaStreamSynchronize(ctx->stream));
    spstd_status ds = check_device_status(ctx);
    if (ds != SPSTD_OK) return ds;
    const int64_t nout = std::min(kept, cap);
    const int64_t first = ctx->steps_taken - nout;  // global index of the first sample returned
    for (int64_t i = 0; i < nout; ++i) {
        const double2 v = row[(first + i) % C];
        re[i] = v.x;
        im[i] = v.y;
    }
    *len = nout;
    return SPSTD_OK;
}

spstd_status spstd_spectrum(spstd_ctx *ctx, int p, int64_t nfft, int max_peaks, double thresh, int phase_correct,
                            double *E, double *amp, int *npeaks)
{
    if (!ctx || !E || !amp || !npeaks) return SPSTD_EINVAL;
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
    double h[3];
    SPSTD_CU(ctx, cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPSTD_CU(ctx, cudaStreamSynchronize(s));
    spstd_status ds = check_device_status(ctx);
    if (ds != SPSTD_OK) return ds;
    double dV = 1.0;
    for (int a = 0; a < ctx->cfg.dims; ++a) dV *= axis_spacing(ctx->cfg, a);
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
    return download_field<T>(ctx, tmp, out);
}
}  // namespace

extern "C" {

spstd_status spstd_energy_norm(spstd_ctx *ctx, double *norm, double *energy)
{
    if (!ctx || !norm || !energy) return SPSTD_EINVAL;
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
constexpr size_t kBatchBytesPerMember = 8192;

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
bool group_uses_tma(const BatchGroupND &g, int ax, int v) { return v == 0 && g.tma[ax]; }

// Blocks per member of a batched pass of axis ax under schedule v (4: the
// plain default where 0 is the TMA pass).
template <typename T>
int group_tiles(const BatchGroupND &g, int ax, int v)
{
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
            if (!a) return prepare_pass_tmared_batch(ax, N, g.n[0], red_planes(g.n, ax));
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
            ta.axis = ax;
            return launch_pass_tmared_batch(ax, N, ta, s);
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
    g.fxy = any && g.tma[0] && g.tma[1];
    for (int i = 0; i < M && g.fxy; ++i) g.fxy = b->slots[g.slots[i]]->fxy_ok && b->slots[g.slots[i]]->fxy_on;
    if (any) {
        std::vector<TmaMember> tm(M);
        for (int i = 0; i < M; ++i) {
            spstd_ctx *ctx = b->slots[g.slots[i]];
            TmaMember &t = tm[i];
            std::memset(&t, 0, sizeof(t));
            for (int f = 0; f < 4; ++f)
                if (g.tma[0]) t.x[f] = ctx->xrmap[f];
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

// ---- autotuner ---------------------------------------------------------------
namespace {

// Schedules an axis of this context can run (sched.h): 0 always; 1..3 for
// plain FFT passes of tunable length; 4 and 5 where 0 is the pipelined TMA pass.
int schedule_candidates(const spstd_ctx *ctx, int ax, int *list)
{
    int n = 0;
    list[n++] = 0;
    if (ax < 0 || ax >= ctx->cfg.dims || ctx->dense[ax] || (ax == 0 && ctx->long_x)) return n;
    const int N = (int)ctx->cfg.n[ax];
    for (int v = 1; v <= 3; ++v) {
        const bool ok = ctx->cfg.precision == 32 ? sched_valid<float>(ax, N, v) : sched_valid<double>(ax, N, v);
        if (ok) list[n++] = v;
    }
    if (ctx->tma[ax]) list[n++] = 4;
    if (ctx->tma[ax] && ctx->tma_st[ax]) list[n++] = 5;
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

// Times the batched passes of one member shape under each schedule on the
// members' scratch fields and keeps the fastest per axis.
template <typename T>
spstd_status tune_group(spstd_batch *b, BatchGroupND &g, int reps, cudaEvent_t e0, cudaEvent_t e1)
{
    const int M = (int)g.slots.size();
    const size_t off = (b->img_bytes + 255) & ~size_t(255);
    if (M == 0 || off + sizeof(PassArgs<T>) * (size_t)M > b->ws_bytes) return SPSTD_OK;  // no room: defaults
    PassArgs<T> *dargs = (PassArgs<T> *)(b->ws + off);
    std::vector<PassArgs<T>> args(M);
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
        for (int v = 0; v <= 4; ++v) {
            if (v >= 1 && v <= 3 && !sched_valid<T>(ax, (int)g.n[ax], v)) continue;
            if (v == 4 && !g.tma[ax]) continue;
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
    if (!fused_active(ctx) && ctx->tma[0] && ctx->sched[0] == 0) {
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
    if (ms)
        for (int i = 0; i < 3 * kSchedules; ++i) ms[i] = -1.0;
    return ctx->cfg.precision == 32 ? tune_impl<float>(ctx, reps, ms) : tune_impl<double>(ctx, reps, ms);
}

spstd_status spstd_batch_tune(spstd_batch *b, int reps)
{
    if (!b || reps < 1) return SPSTD_EINVAL;
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
