/*
 * spstd.h -- C ABI of the GB300 (sm_103a) SPSTD library.
 *
 * The library advances the time-dependent Schroedinger equation
 *     i hbar d psi/dt = -(hbar^2/2m*) lap psi + V(r) psi            (Eq. 1)
 * split into the real fields psi = psi_R + i psi_I (Eq. 2-4), with the
 * symplectic pseudospectral time-domain (SPSTD) scheme of arXiv 1805.03155:
 * spatial second derivatives by FFT (Eq. 7-10) and an m-stage partitioned
 * symplectic product in time (Eq. 14-18).  Eigen-energies are read off the
 * spectrum of probe-point time series (Tables 2-4).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an spstd_status; nothing throws across the ABI.
 *  - Grids are periodic boxes [lo_d, hi_d) with n_d points per axis,
 *    x_j = lo + j (hi - lo)/n (Eq. 5/6).  Field arrays are [n2][n1][n0] with
 *    axis 0 (x) fastest; unused axes have n = 1.
 *  - Host arrays are owned by the caller and only read or written during the
 *    call (set_* copy in, get_* copy out).
 *  - Device memory: the caller allocates ONE device buffer of
 *    spstd_workspace_size() bytes (256-byte aligned) and hands it to
 *    spstd_create(); the library carves all its device state from it and never
 *    allocates device memory itself.  The buffer must outlive the context.
 *  - All device work is enqueued on cfg.stream (NULL = the legacy default
 *    stream).  spstd_step() returns without waiting; the calls that return
 *    host results (get_state, probe, spectrum, energy_norm,
 *    apply_hamiltonian) synchronise that stream.
 *  - A context is not thread safe; distinct contexts are independent.
 *  - On error the context keeps its previous state where possible and
 *    spstd_last_error() describes the failure.
 */
#ifndef SPSTD_H
#define SPSTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spstd_ctx spstd_ctx;
typedef struct spstd_batch spstd_batch;

typedef enum {
    SPSTD_OK = 0,
    SPSTD_EINVAL = 1,       /* bad argument (NULL, size out of range, bad index) */
    SPSTD_ENOMEM = 2,       /* workspace too small, or host allocation failed */
    SPSTD_ECUDA = 3,        /* a CUDA runtime call failed (message in last_error) */
    SPSTD_EUNSTABLE = 4,    /* dt above the stability limit s_star/w_max (Eq. 25/30) */
    SPSTD_EDIVERGED = 5,    /* norm or energy is NaN/Inf, or the norm drifted past cfg.norm_drift_limit */
    SPSTD_ETIMEOUT = 6,     /* a bounded device wait gave up (reported at the next synchronising call) */
    SPSTD_ENOTREADY = 7,    /* nothing to return yet (no probe samples) */
    SPSTD_EUNSUPPORTED = 8  /* valid request this build does not implement */
} spstd_status;

/* Integrator presets for Eq. 17 (coefficients c_l, d_l, l = 1..m).
 *  SPSTD_LEAPFROG  m = 1, c = d = 1: the traditional explicit PSTD update
 *                  (Eq. 11/12), order 1 in this partitioned form.
 *  SPSTD_STRANG    m = 2, c = (1/2, 1/2), d = (1, 0): order 2.
 *  SPSTD_PAPER3    the paper's set (after Eq. 18): c = (0.26833010,
 *                  -0.18799162, 0.91966152), d_l = c_{m-l+1}.
 *  SPSTD_FR4       Yoshida triple jump of the Strang step (order 4),
 *                  x = 1/(2 - 2^(1/3)): c = (x/2, (1-x)/2, (1-x)/2, x/2),
 *                  d = (x, 1-2x, x, 0).
 *  SPSTD_SUZUKI6   Suzuki five-fold Strang composition (order 4),
 *                  p = 1/(4 - 4^(1/3)): c = (p/2, p, (1-3p)/2, (1-3p)/2, p, p/2),
 *                  d = (p, p, 1-4p, p, p, 0).
 *  SPSTD_CUSTOM    use cfg.m, cfg.c, cfg.d as given (m <= 8).
 *  SPSTD_RK4       not symplectic: the classical fourth-order Runge-Kutta
 *                  scheme the paper compares against (Fig. 3), on the same
 *                  kernels (8 K applications per step); stable for w dt <= 2 sqrt 2. */
enum {
    SPSTD_CUSTOM = -1,
    SPSTD_LEAPFROG = 0,
    SPSTD_STRANG = 1,
    SPSTD_PAPER3 = 2,
    SPSTD_FR4 = 3,
    SPSTD_SUZUKI6 = 4,
    SPSTD_RK4 = 5
};

#define SPSTD_MAX_STAGES 8
#define SPSTD_MAX_PROBES 16
#define SPSTD_MAX_EIGENSTATES 4

typedef struct {
    int dims;             /* 1, 2 or 3 */
    int64_t n[3];         /* points per axis, x first.  Each used axis: a power
                             of two (periodic), 2 <= n <= 4194304 for x and
                             2 <= n <= 1024 for y and z, or any 2 <= n <= 256
                             (see bc below); unused axes: 1.  x lines longer
                             than one block transforms (8192 FP32 / 4096 FP64
                             in 1D, 1024 otherwise) take a four-step FFT
                             through a scratch array in the workspace */
    double lo[3], hi[3];  /* periodic box per axis, hi > lo */
    double hbar, mass;    /* hbar and effective mass m* (> 0) */
    int precision;        /* 32 or 64: type of the fields and of the FFTs;
                             reductions and spectra are FP64 in both */
    int preset;           /* SPSTD_* preset id, or SPSTD_CUSTOM */
    int m;                /* SPSTD_CUSTOM only: stages (1..8) */
    double c[SPSTD_MAX_STAGES], d[SPSTD_MAX_STAGES]; /* SPSTD_CUSTOM only */
    double dt;            /* time step; <= 0 selects half the stability limit */
    int n_probe;          /* 0..16 probe points */
    int64_t probe_idx[SPSTD_MAX_PROBES]; /* flat grid index of each probe */
    int64_t probe_capacity; /* samples kept per probe (ring buffer), >= 1 */
    int64_t max_nfft;     /* largest spectrum length (power of two); <= 0
                             selects next_pow2(4 * probe_capacity) */
    int nyquist_zero;     /* 0: k^2 = (pi/dx)^2 at the Nyquist index (default);
                             1: Nyquist mode zeroed (literal Eq. 10) */
    int device;           /* CUDA device ordinal the workspace lives on */
    void *stream;         /* cudaStream_t for all work; NULL = legacy default */
    int bc[3];            /* per axis boundary (Section 2.2): SPSTD_PERIODIC (DFT),
                             SPSTD_DIRICHLET (DST, n interior points between walls
                             at lo and hi) or SPSTD_NEUMANN (DCT, n points including
                             both walls) */
    int max_eigenstates;  /* 0..4: eigenstate accumulators to reserve (FP64 complex,
                             16 B per grid point each) */
    int unmerged_steps;   /* 0 (default): when the last half-stage of a step and
                             the first of the next update the same field (FR4,
                             SUZUKI6, STRANG), consecutive steps of one spstd_step
                             call apply them as one half-stage with the summed
                             coefficient -- exact, since both act with the other
                             field unchanged (Eq. 17: exp(aA) exp(bA) =
                             exp((a+b)A)); the probe at that step boundary is
                             recovered exactly from the fields before and after.
                             1: always run every half-stage of every step. */
    int no_graph;         /* 0 (default): spstd_step replays captured CUDA graphs
                             of 16-step units; 1: it launches every kernel
                             directly.  Both enqueue the same kernels with the
                             same arguments in the same order, so the results
                             are the same bits (a check of the replay). */
    double norm_drift_limit; /* divergence rule: spstd_energy_norm returns
                             SPSTD_EDIVERGED (after writing its outputs) when
                             |N / N0 - 1| exceeds this, N0 being the norm of the
                             state last given to spstd_set_state.  The schemes
                             of Eq. 17 conserve the norm to rounding (a bounded
                             oscillation), so a larger drift means an unstable
                             dt or corrupted fields.  spstd_config_init sets
                             1e-3; <= 0 turns the check off (e.g. for the RK4
                             comparison, whose norm decays by design). */
    int v_field_only;     /* 0 (default): an FP32 grid whose potential separates,
                             V(x, y, z) = vx(x) + vyz(y, z) to 4 units in the
                             last place, gets the two FP32 tables, and the V
                             field holds their FP32 sums; the reduce-add x passes
                             (single grid and batched) then rebuild the V term
                             from the tables (12 instead of 16 B per point) with
                             the same bits.  1: every pass reads the V field
                             (Eq. 16's V at every point, as for any potential). */
} spstd_config;

/* Boundary conditions (Section 2.2).  Periodic axes whose length is a power of
 * two use the FFT passes; wall axes, and periodic axes of any other length
 * 2 <= n <= 256, apply the same spectral operator as a dense n x n matrix
 * (FP64-built, rounded once), which for such short lines costs no more than the
 * transforms.  On FP32 2D/3D grids, axes of 32..128 points apply it on the
 * tensor cores as one product over all lines (TF32 with the 3xTF32 split, FP32
 * accumulation: FP32 accuracy, not the CUDA-core sum's exact rounding).  Grid points: periodic x_j = lo + j L/n; Dirichlet
 * x_j = lo + (j+1) L/(n+1); Neumann x_j = lo + j L/(n-1). */
enum { SPSTD_PERIODIC = 0, SPSTD_DIRICHLET = 1, SPSTD_NEUMANN = 2 };
#define SPSTD_MAX_DENSE_N 256

/* Fills cfg with defaults: dims 1, n = (256, 1, 1), box [0, 1), hbar = m* = 1,
 * precision 64, SPSTD_FR4, dt = 0 (auto), no probes, capacity 1024. */
void spstd_config_init(spstd_config *cfg);

/* Bytes of device workspace a context for cfg needs.  Validates cfg
 * (SPSTD_EINVAL / SPSTD_EUNSUPPORTED / SPSTD_EUNSTABLE as spstd_create). */
spstd_status spstd_workspace_size(const spstd_config *cfg, size_t *bytes);

/* Stability of the configured scheme (Eq. 23-25, Table 1): s_star is the
 * largest s with |tr M(s')| <= 2 for all 0 <= s' <= s, M the per-mode step
 * matrix; dt_max = s_star / w_max with the Weyl bound
 * w_max = (hbar/2m*) sum_d (pi/dx_d)^2 + max(V, 0)/hbar, using vmax for max V. */
spstd_status spstd_stability_limit(const spstd_config *cfg, double vmax, double *s_star,
                                   double *dt_max);

/* Creates a context on the caller's workspace (device pointer, 256-byte
 * aligned, >= spstd_workspace_size bytes).  Uploads the FFT twiddles and the
 * per-stage k^2 multipliers (both computed in FP64 and rounded to the field
 * precision once).  Fields start at zero, V at zero.  If cfg.dt <= 0 the time
 * step is chosen at set_potential time as half the stability limit.
 * *out is NULL on failure. */
spstd_status spstd_create(const spstd_config *cfg, void *d_workspace, size_t workspace_bytes,
                          spstd_ctx **out);

/* Releases the host side of the context (the workspace stays the caller's).
 * Waits for the context's stream first.  NULL is accepted. */
spstd_status spstd_destroy(spstd_ctx *ctx);

/* Copies V (host, FP64, n_total values, x fastest) to the device, rounded to
 * the field precision.  Re-derives dt when cfg.dt <= 0 and re-checks the
 * stability limit (SPSTD_EUNSTABLE if a fixed dt is above it).
 *
 * Separable potentials (FP32 fields, 2D/3D, x axis of 32..512 points): when
 * V(x, y, z) = vx(x) + vyz(y, z) with FP32 tables whose FP32 sum is within 4
 * units in the last place of every value of V (the split is taken at the
 * point of smallest |V|, so wells of one sign qualify), the device V holds
 * those sums instead of V rounded to FP32, and the x pass rebuilds the V term
 * (Eq. 16's V/hbar psi) from the two tables instead of reading the V field:
 * 12 instead of 16 bytes of HBM traffic per point in that pass.  Waits for
 * the context's stream in that case (the tables are copied from host memory
 * that is freed on return). */
spstd_status spstd_set_potential(spstd_ctx *ctx, const double *V);

/* *separable = 1 if the x pass rebuilds the V term from separable tables
 * (see spstd_set_potential), else 0. */
spstd_status spstd_potential_separable(const spstd_ctx *ctx, int *separable);

/* Host only (no device work, no context): the split spstd_set_potential
 * tries.  V: host, nx * rows values, x fastest (rows = ny nz).  vx (nx floats)
 * and vyz (rows floats) are caller-owned outputs.  *separable = 1 when the
 * FP32 sum vx[i] + vyz[r] is within 4 units in the last place of
 * V[r nx + i] at every point (the tables are then the ones the x pass uses),
 * else 0 (vx and vyz then hold the rejected split).  SPSTD_EINVAL for null
 * pointers or nx, rows < 1. */
spstd_status spstd_separable_split(const double *V, int64_t nx, int64_t rows, float *vx, float *vyz,
                                   int *separable);

/* Copies the state (host, FP64, n_total values each) to the device and resets
 * the probe recorder (step counter 0, no samples).  The norm N0 of the
 * divergence rule is summed on the device from these FP64 values; the next
 * spstd_energy_norm reads it back.  Enqueued on cfg.stream: pageable host
 * arrays are read before the call returns; pinned (page-locked) ones are read
 * by the copies as the stream reaches them, so they must not change until
 * then. */
spstd_status spstd_set_state(spstd_ctx *ctx, const double *psiR, const double *psiI);

/* Copies the current state to the host as FP64 (synchronises). */
spstd_status spstd_get_state(spstd_ctx *ctx, double *psiR, double *psiI);

/* Enqueues nsteps full steps of Eq. 17/18: for l = 1..m,
 *     psi_R += c_l dt K psi_I,  then  psi_I -= d_l dt K psi_R,
 * K = -(hbar/2m*) lap + V/hbar (Eq. 16), zero coefficients skipped, and after
 * every step records psi_R + i psi_I at each probe.  nsteps = 0 is a no-op.
 * Asynchronous; repeated chunks are replayed from a captured CUDA graph (2D
 * and 3D grids), which the first call on a context captures whatever its
 * length (and the first call after a change of schedule or potential). */
spstd_status spstd_step(spstd_ctx *ctx, int64_t nsteps);

/* Copies the recorded series of probe p (0 <= p < n_probe), oldest first,
 * FP64: up to cap samples (the most recent ones if more were kept); *len gets
 * the count.  SPSTD_ENOTREADY if no step has been recorded. */
spstd_status spstd_probe(spstd_ctx *ctx, int p, double *re, double *im, int64_t cap,
                         int64_t *len);

/* Eigen-energies from the spectrum of probe p's series (p = -1: the sum of all
 * probes), computed on the device in FP64: symmetric Hann window, zero padding
 * to nfft (power of two, M <= nfft <= max_nfft; <= 0 picks next_pow2(4M)),
 * peaks among positive energies that are the largest value within the
 * window's main-lobe half width ceil(2 nfft/M) bins and >= thresh * the
 * largest, the max_peaks largest kept, each refined by 60 golden-section
 * steps on the windowed DTFT.  E = hbar theta/dt; with phase_correct != 0 the
 * map's dispersion is inverted (theta = arccos(tr M(w dt)/2) solved for w) and
 * E = hbar w.  Outputs sorted by E ascending: E[i], amp[i] (DTFT magnitude
 * over the window sum), *npeaks <= max_peaks.  Synchronises. */
spstd_status spstd_spectrum(spstd_ctx *ctx, int p, int64_t nfft, int max_peaks, double thresh,
                            int phase_correct, double *E, double *amp, int *npeaks);

/* Workspace canaries (a debugging aid: the GPU memory checker is not always
 * available).  The workspace holds 256 guard bytes of a fixed pattern after
 * each of its regions (fields, tables, rings, scratch); spstd_check_workspace
 * reads them back after the work enqueued so far (it synchronises the
 * context's stream) and sets *intact to 0 if any was overwritten -- a kernel
 * wrote past the end of its region -- naming the first in spstd_last_error.
 * The guards are not written again: a damaged workspace stays reported. */
spstd_status spstd_check_workspace(spstd_ctx *ctx, int *intact);

/* norm = dV sum(psi_R^2 + psi_I^2) and energy = dV sum(psi_R H psi_R +
 * psi_I H psi_I), H = hbar K, accumulated in FP64 on the device in a fixed
 * order (bitwise reproducible).  Synchronises.  SPSTD_EDIVERGED if either is
 * not finite (the values are still written). */
spstd_status spstd_energy_norm(spstd_ctx *ctx, double *norm, double *energy);

/* out = H psi_which (which 0: psi_R, 1: psi_I) as FP64 on the host, computed by
 * the same FFT pass kernels as a step.  Synchronises. */
spstd_status spstd_apply_hamiltonian(spstd_ctx *ctx, int which, double *out);

/* The time step in use, the steps taken since set_state, the integrator. */
spstd_status spstd_get_dt(const spstd_ctx *ctx, double *dt);
spstd_status spstd_steps_taken(const spstd_ctx *ctx, int64_t *steps);
spstd_status spstd_get_coefficients(const spstd_ctx *ctx, int *m, double *c, double *d);

/* Number of kernels spstd_step(ctx, nsteps) runs on the device (kernel nodes
 * of replayed graphs included). */
spstd_status spstd_launch_count(const spstd_ctx *ctx, int64_t nsteps, int64_t *launches);

/* Per-kernel timing: runs nsteps steps (real steps: the state advances and the
 * probes record) with direct launches instead of graph replays, a CUDA event
 * pair around every launch on the context's stream, and returns per kernel
 * kind k the summed device time ms[k] (milliseconds) and launch count cnt[k]:
 * k = 0 x pass, 1 y pass, 2 z pass, 3 probe recorder, 4 resident 1D solver,
 * 5 fused x-y pass.  Synchronises. */
#define SPSTD_KERNEL_KINDS 6
spstd_status spstd_profile_steps(spstd_ctx *ctx, int64_t nsteps, double *ms, int64_t *cnt);

/* Schedules: the radix and tile plan of an axis's pass kernel (no effect on
 * what is computed; Eq. 10's transform in a different shape).
 *   0  the axis's default kernel (the pipelined TMA pass for FP32 2D/3D axes
 *      of 32..512 points, whose destination field is accumulated at L2 by a
 *      TMA reduce-add, else the plain pass: 16 FP32 / 8 FP64 points per
 *      thread, about 256 threads per block)
 *   1  plain pass, half the lines per block
 *   2  plain pass, twice the lines per block
 *   3  plain pass, half the points per thread (one radix lower per stage)
 *   4  plain pass, default plan (listed only where 0 is the TMA pass); on a
 *      dense wall axis whose 0 is the tensor-core product (FP32 2D/3D, 32..128
 *      points): the CUDA-core dense pass
 *   5  TMA pass that loads the destination tile into shared memory, adds
 *      there and stores it back (listed only where 0 is the TMA pass)
 *   6  x axes of 32, 48, 64, 96, 128 or 256 points of FP32 2D/3D grids
 *      (single and batched): the reduce-add TMA pass with per-warp tiles
 *      (each warp its own ring of stages and barriers); the same arithmetic
 *      as 0, so the same bits
 * Schedules 1..3 exist for FFT axes of 32..512 points.  0, 1, 2 and 4 give
 * bit-identical results on plain axes; 3 changes the rounding (FP32 ~1e-7).
 * spstd_schedule_candidates lists the schedules axis (0..dims-1) can run in
 * list[0..*count) (list holds SPSTD_SCHEDULES ints).  spstd_set_schedule
 * selects one (SPSTD_EINVAL if not a candidate); the next step re-captures its
 * graph.  spstd_tune times every candidate of every axis on this context's
 * grid -- H applied to psi_I into the scratch field, once to warm up then reps
 * times, on the context's stream -- keeps the fastest per axis and, when ms is
 * not NULL, writes the mean milliseconds per pass to ms[axis * SPSTD_SCHEDULES
 * + schedule] (-1 where not a candidate).  It synchronises and leaves psi_R,
 * psi_I, the probes and the step count unchanged. */
#define SPSTD_SCHEDULES 7
spstd_status spstd_schedule_candidates(const spstd_ctx *ctx, int axis, int *list, int *count);
spstd_status spstd_get_schedule(const spstd_ctx *ctx, int axis, int *schedule);
spstd_status spstd_set_schedule(spstd_ctx *ctx, int axis, int schedule);
spstd_status spstd_tune(spstd_ctx *ctx, int reps, double *ms);

/* x-y fusion.  Two fused forms of a half-stage's x and y passes exist, both
 * for FP32 grids with x and y on schedule 0 (Eq. 18's x and y terms summed in
 * one launch; FP32 rounding differs from the separate passes):
 *  - the reduce-add fused pass, for nx = ny in {32, 64} (3D; 2D at 64): a
 *    unit of planes holds whole x and whole y lines in shared memory, both
 *    transforms run on it and one reduce-add writes x + y + V terms.  On by
 *    default where it applies;
 *  - the stored-tile fused pass (3D, nx = ny in {64, 128, 256}; off by
 *    default): one persistent launch visits every plane's y tiles and then,
 *    while the plane is still in L2, its x tiles.
 * spstd_set_xy_fusion turns the stored-tile form on or off (it takes
 * precedence) and returns SPSTD_EUNSUPPORTED for a grid that cannot use it;
 * *on reports whether steps use it.  spstd_tune times separate passes and each
 * fused form that applies and keeps the fastest. */
spstd_status spstd_set_xy_fusion(spstd_ctx *ctx, int on);
spstd_status spstd_get_xy_fusion(const spstd_ctx *ctx, int *on);


/* Norm without device allocation (the paper has no counterpart: this is a
 * service for callers that may not allocate device memory where they call).
 * Computes *d_norm = cell_volume * sum_i (psiR[i]^2 + psiI[i]^2) in FP64, in a
 * fixed order, from n values of psiR and psiI (device pointers, FP32 or FP64
 * per precision, caller-owned) into d_norm (a device double, caller-owned),
 * enqueued on stream (cudaStream_t; NULL = legacy default) without waiting.
 * Its per-block partial sums live in a static device array of
 * SPSTD_NOALLOC_MAX_PARTIALS doubles (512 KB on every GPU that loads the
 * library, kept until the process exits) instead of caller memory; it calls no
 * cudaMalloc, cudaFree or allocating library routine.  Every call on a device
 * shares that array: calls that overlap on the GPU race and must be
 * serialised (e.g. one stream).  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  The address is kept per
 * device ordinal for the life of the process, so the entry point assumes the
 * CUDA runtime's primary context on each device: do not call it from another
 * (driver-API) context on the same device, nor after cudaDeviceReset.  SPSTD_EINVAL for NULL
 * pointers, n <= 0, a bad precision, or n > SPSTD_NOALLOC_MAX_ELEMS;
 * SPSTD_ECUDA if the set-up or a launch fails. */
#define SPSTD_NOALLOC_MAX_PARTIALS 65536
#define SPSTD_NOALLOC_MAX_ELEMS ((int64_t)SPSTD_NOALLOC_MAX_PARTIALS * 2048)
spstd_status spstd_norm_noalloc(const void *psiR, const void *psiI, int64_t n, int precision,
                                double cell_volume, double *d_norm, void *stream);

/* ---- Eigenstates (Figs. 1, 2, 4: the eigenstate of a spectral peak) -------
 * spstd_eigenstates_begin opens an accumulation window: each of the next
 * `window` steps adds, for every target energy E_k (k < n_target <=
 * cfg.max_eigenstates), w_n psi^n exp(+i E_k t_n / hbar) to accumulator k at
 * every grid point (FP64), with w_n the symmetric Hann window over the window
 * and t_n the time after the n-th step of the window.  The result is the
 * eigenstate at E_k up to normalisation and phase (components at other
 * energies are suppressed by the window).  While a window is open steps run
 * without fused boundaries or the resident 1D solver (every step ends at a
 * full state).  spstd_eigenstate_get copies accumulator k to the caller's
 * host arrays re, im (n_total doubles each) and synchronises; with normalise =
 * 0 they hold the raw accumulator, with normalise = 1 it is scaled to
 * sum |phi|^2 = 1 and its phase turned so that its largest-modulus entry (the
 * first, if several) is real and positive -- the form in which eigenstates are
 * compared and plotted (Figs. 1, 2, 4); an all-zero accumulator stays zero.
 * *samples (may be NULL) receives the steps accumulated so far.
 * spstd_eigenstates_end closes the window. */
spstd_status spstd_eigenstates_begin(spstd_ctx *ctx, int n_target, const double *E, int64_t window);
spstd_status spstd_eigenstate_get(spstd_ctx *ctx, int k, int normalise, double *re, double *im, int64_t *samples);
spstd_status spstd_eigenstates_end(spstd_ctx *ctx);

/* ---- Batches: many independent solves advanced by one call ---------------
 * A batch advances every member context by the same number of steps, each with
 * its own grid, V, dt, integrator and probes.  1D members of one length run all
 * steps of a call in one resident block each (one launch per length); 2D/3D
 * members that share dims, sizes, precision and integrator run every pass of
 * every half-stage as one launch over all their tiles; the 2D/3D groups follow
 * one another in a captured CUDA graph, replayed in chunks, while the 1D
 * resident launches run beside them on a second stream.  Results equal those
 * of stepping each member alone up to FP rounding order (bit for bit where
 * the batch and the lone member run the same pass kernels and plans).
 * Members stay usable (get_state, probe, spectrum, energy_norm) between batch
 * steps; do not call spstd_step on a member while it is in a batch.
 * Device memory: one caller-owned workspace of spstd_batch_workspace_size()
 * bytes (256-byte aligned) for the member descriptors. */
typedef struct spstd_batch spstd_batch;
spstd_status spstd_batch_workspace_size(int max_members, size_t *bytes);
/* stream: cudaStream_t for all batch work (NULL = legacy default stream);
 * device: the CUDA device every member lives on.  hbm_cap_bytes: admission by
 * device footprint -- the members' workspaces (spstd_workspace_size of each
 * member's config) may sum to at most this many bytes; 0 = no cap. */
spstd_status spstd_batch_create(int max_members, size_t hbm_cap_bytes, int device, void *stream,
                                void *d_workspace, size_t workspace_bytes, spstd_batch **out);
spstd_status spstd_batch_destroy(spstd_batch *b);
/* Admits ctx as a member (waits for ctx's own stream first); *slot receives
 * its index.  SPSTD_ENOTREADY when the batch is full or the member's workspace
 * would take the batch over its HBM cap (retry after a removal);
 * SPSTD_EINVAL if ctx is already in a batch, lives on another device or alone
 * exceeds the cap; SPSTD_EUNSUPPORTED for members a batch cannot step (wall or
 * dense axes, long lines, RK4). */
spstd_status spstd_batch_add(spstd_batch *b, spstd_ctx *ctx, int *slot);
/* Retires the member in slot after the batch stream has drained; its
 * footprint leaves the batch's total. */
spstd_status spstd_batch_remove(spstd_batch *b, int slot);
/* Bytes of member workspaces admitted now, and the cap (0 = none). */
spstd_status spstd_batch_footprint(const spstd_batch *b, size_t *in_use, size_t *cap);
spstd_status spstd_batch_size(const spstd_batch *b, int *members);
/* Enqueues nsteps steps of every member on the batch stream (asynchronous). */
spstd_status spstd_batch_step(spstd_batch *b, int64_t nsteps);
/* Waits for the batch stream. */
spstd_status spstd_batch_sync(spstd_batch *b);
/* Kernel launches one spstd_batch_step(b, nsteps) runs (graph nodes included). */
spstd_status spstd_batch_launch_count(const spstd_batch *b, int64_t nsteps, int64_t *launches);
const char *spstd_batch_last_error(const spstd_batch *b);
/* Autotunes the batched passes: for every 2D/3D member shape and axis, times
 * the batched pass under schedules 0..4 and 6 over all members of that shape
 * (0 = the default: the pipelined TMA reduce-add pass over every member's
 * tiles for FP32 axes of 32..512, 48 or 96 points, else the plain plan; 1..3 as
 * for a lone context; 4 = the plain plan where 0 is the TMA pass; 6 = the x
 * pass on per-warp tiles, for x lines where a lone context lists it) -- H
 * applied into each member's scratch field, once to warm up then reps times --
 * and keeps the fastest.  The choice is kept per
 * shape (precision, dims, n) for as long as the batch lives, including members
 * added later; the states are not touched.  Synchronises the batch stream. */
spstd_status spstd_batch_tune(spstd_batch *b, int reps);
/* The batch's schedules for a member shape (0 where not tuned); n: 3 sizes. */
spstd_status spstd_batch_get_schedule(const spstd_batch *b, int precision, int dims, const int64_t *n, int *schedule);
/* Sets the schedules of a 2D/3D member shape (precision 32/64, dims, n: 3
 * sizes, schedule: dims values) as spstd_batch_tune would, for members present
 * and added later; the batch re-captures its graph at the next step.  Allowed
 * per axis: 0, 4, 1..3 where a lone context of that shape lists them, and 6 on
 * the x axis of FP32 shapes whose x lines take per-warp tiles (a group whose
 * members lack those maps runs 0 instead).  SPSTD_EINVAL otherwise. */
spstd_status spstd_batch_set_schedule(spstd_batch *b, int precision, int dims, const int64_t *n, const int *schedule);

/* Human-readable text of the last failure on ctx (never NULL). */
const char *spstd_last_error(const spstd_ctx *ctx);
const char *spstd_status_string(spstd_status s);

#ifdef __cplusplus
}
#endif
#endif /* SPSTD_H */
