/*
 * spstd_oracle.c -- plain FP64 CPU oracle for the SPSTD method of
 * arXiv 1805.03155 (symplectic pseudospectral time domain for the TDSE).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  It shares no code
 * with the CUDA library.  Slow and obvious on purpose: no blocking, no line
 * pairing, no fusion.  Each function names the passage it follows.
 *
 * Readings of the paper taken here (each is pinned by a test, see tests/):
 *  - Eq. 16/17: the state is advanced stage by stage, l = 1..m; inside a stage
 *    the A factor (psi_R += c_l dt K psi_I) acts first, then the B factor
 *    (psi_I -= d_l dt K psi_R) using the new psi_R.
 *  - Eq. 10: the second derivative is applied as one multiply by -K_n^2 in
 *    Fourier space.  At the Nyquist index of an even grid k^2 = (pi/dx)^2 is
 *    kept unless the grid asks for it to be zeroed (the literal reading of
 *    Eq. 10, which keeps only real parts after each inverse transform).
 *  - Eq. 22/23/26/29 print k where k^2 is meant: the per-mode rate is
 *    w = hbar |k|^2 / 2m* (+ V/hbar for a potential eigenmode).
 */
#include "spstd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double TWO_PI = 6.28318530717958647692528676655900577;

/* ------------------------------------------------------------------------ */
/* Integrator coefficients (Eq. 17; the paper's own set is printed after     */
/* Eq. 18 and again after Eq. 30).                                           */
/* ------------------------------------------------------------------------ */

/* Fills c[0..m), d[0..m) for a preset.  Returns 0 on success, -1 on an unknown
 * id.
 *  LEAPFROG: m = 1, c = d = 1 (the traditional explicit PSTD update, Eq. 11/12).
 *  STRANG:   m = 2, c = (1/2, 1/2), d = (1, 0).
 *  PAPER3:   the set printed after Eq. 18: c = (0.26833010, -0.18799162,
 *            0.91966152), d_l = c_{m-l+1}.
 *  FR4:      Yoshida's triple jump of the Strang step, x = 1/(2 - 2^(1/3)):
 *            c = (x/2, (1-x)/2, (1-x)/2, x/2), d = (x, 1-2x, x, 0).
 *  SUZUKI6:  Suzuki's five-fold Strang composition with p = 1/(4 - 4^(1/3))
 *            and weights (p, p, 1-4p, p, p): c = (p/2, p, (1-3p)/2,
 *            (1-3p)/2, p, p/2), d = (p, p, 1-4p, p, p, 0). */
int orc_preset(int id, double *c, double *d, int *m)
{
    if (id == ORC_LEAPFROG) {
        *m = 1; c[0] = 1.0; d[0] = 1.0;
        return 0;
    }
    if (id == ORC_STRANG) {
        *m = 2; c[0] = 0.5; c[1] = 0.5; d[0] = 1.0; d[1] = 0.0;
        return 0;
    }
    if (id == ORC_PAPER3) {
        *m = 3;
        c[0] = 0.26833010; c[1] = -0.18799162; c[2] = 0.91966152;
        for (int l = 0; l < 3; ++l) d[l] = c[3 - 1 - l];
        return 0;
    }
    if (id == ORC_FR4) {
        double x = 1.0 / (2.0 - cbrt(2.0));
        *m = 4;
        c[0] = x / 2; c[1] = (1 - x) / 2; c[2] = (1 - x) / 2; c[3] = x / 2;
        d[0] = x; d[1] = 1 - 2 * x; d[2] = x; d[3] = 0.0;
        return 0;
    }
    if (id == ORC_SUZUKI6) {
        double p = 1.0 / (4.0 - cbrt(4.0));
        *m = 6;
        c[0] = p / 2; c[1] = p; c[2] = (1 - 3 * p) / 2; c[3] = (1 - 3 * p) / 2; c[4] = p; c[5] = p / 2;
        d[0] = p; d[1] = p; d[2] = 1 - 4 * p; d[3] = p; d[4] = p; d[5] = 0.0;
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* FFT (the "fast Fourier transform" used for Eq. 8/9): recursive decimation */
/* in time, radix 2 and 3, direct sum for any other prime factor.            */
/* ------------------------------------------------------------------------ */

/* out[0..n) = DFT_n of in[0], in[s], ..., in[(n-1)s].  W[k] = exp(-2 pi i k/Wn)
 * for k < Wn and n divides Wn.  sign < 0: exp(-...) (forward), sign > 0:
 * exp(+...) (inverse, unnormalised). */
static void dft_rec(const double complex *in, int64_t s, double complex *out, int64_t n,
                    const double complex *W, int64_t Wn, int sign)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int64_t step = Wn / n; /* W[e*step] = exp(-2 pi i e / n) */
    int64_t r = (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : n;
    if (r == n) {
        for (int64_t k = 0; k < n; ++k) {
            double complex acc = 0;
            for (int64_t j = 0; j < n; ++j) {
                double complex w = W[((j * k) % n) * step];
                if (sign > 0) w = conj(w);
                acc += in[j * s] * w;
            }
            out[k] = acc;
        }
        return;
    }
    int64_t m = n / r;
    /* X[k + p m] = sum_q w_n^{q (k + p m)} Y_q[k],  Y_q = DFT_m(x_q, x_{q+r}, ...) */
    for (int64_t q = 0; q < r; ++q) dft_rec(in + q * s, s * r, out + q * m, m, W, Wn, sign);
    for (int64_t k = 0; k < m; ++k) {
        double complex y[3];
        for (int64_t q = 0; q < r; ++q) y[q] = out[q * m + k];
        for (int64_t p = 0; p < r; ++p) {
            double complex acc = 0;
            for (int64_t q = 0; q < r; ++q) {
                double complex w = W[((q * (k + p * m)) % n) * step];
                if (sign > 0) w = conj(w);
                acc += y[q] * w;
            }
            out[p * m + k] = acc;
        }
    }
}

static double complex *twiddles(int64_t n)
{
    double complex *W = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    if (!W) return NULL;
    for (int64_t k = 0; k < n; ++k) {
        double a = TWO_PI * (double)k / (double)n;
        W[k] = cos(a) - I * sin(a);
    }
    return W;
}

static int fft_with(double complex *x, double complex *tmp, int64_t n, const double complex *W, int sign)
{
    dft_rec(x, 1, tmp, n, W, n, sign);
    memcpy(x, tmp, sizeof(double complex) * (size_t)n);
    return 0;
}

/* In-place unnormalised DFT of (re + i im): sign < 0 gives
 * X_k = sum_j x_j exp(-2 pi i jk/n) (Eq. 8 up to the 1/L factor), sign > 0 the
 * inverse sum without the 1/n factor.  Returns 0, or -1 on bad input. */
int orc_fft(double *re, double *im, int64_t n, int sign)
{
    if (n <= 0 || !re || !im) return -1;
    double complex *x = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    double complex *t = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    double complex *W = twiddles(n);
    if (!x || !t || !W) {
        free(x); free(t); free(W);
        return -1;
    }
    for (int64_t j = 0; j < n; ++j) x[j] = re[j] + I * im[j];
    fft_with(x, t, n, W, sign);
    for (int64_t j = 0; j < n; ++j) {
        re[j] = creal(x[j]);
        im[j] = cimag(x[j]);
    }
    free(x); free(t); free(W);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Spectral second derivative (Eq. 7-10).                                    */
/* ------------------------------------------------------------------------ */

/* k^2 for DFT index j of an n-point axis of period L: K_n = 2 pi n'/L with the
 * wrapped index n' = j (j < n/2) or j - n (Eq. 8: n = 0, +-1, +-2, ...). */
static double k2_of(int64_t j, int64_t n, double L, int nyquist_zero)
{
    if (nyquist_zero && n % 2 == 0 && j == n / 2) return 0.0;
    int64_t w = (j <= n / 2) ? j : j - n;
    double k = TWO_PI * (double)w / L;
    return k * k;
}

/* out = L_axis f = Re F^{-1}[ k^2 F f ] along one axis, i.e. -d^2 f/dx_axis^2
 * (Eq. 10 with the two multiplies by iK folded into one by -K^2).  Every line
 * is transformed on its own, as a complex line with zero imaginary part.
 * Walls (Section 2.2) use the same periodic transform on the line's odd
 * (Dirichlet: the DST) or even (Neumann: the DCT) extension over a period of
 * twice the box, read back on the original points. */
int orc_laplacian_axis(const double *f, double *out, const orc_grid *g, int axis)
{
    if (!f || !out || !g || axis < 0 || axis >= g->dims) return -1;
    const int bc = g->bc[axis];
    int64_t n = g->n[axis];
    int64_t stride = 1, outer = 1;
    for (int b = 0; b < axis; ++b) stride *= g->n[b];
    for (int b = axis + 1; b < 3; ++b) outer *= g->n[b];
    double L = g->hi[axis] - g->lo[axis];
    if (bc == ORC_NEUMANN && n < 2) return -1;
    /* length and period of the line the transform sees */
    int64_t P = bc == ORC_DIRICHLET ? 2 * (n + 1) : bc == ORC_NEUMANN ? 2 * (n - 1) : n;
    double Lp = bc == ORC_PERIODIC ? L : 2.0 * L;
    double complex *x = (double complex *)malloc(sizeof(double complex) * (size_t)P);
    double complex *t = (double complex *)malloc(sizeof(double complex) * (size_t)P);
    double complex *W = twiddles(P);
    if (!x || !t || !W) {
        free(x); free(t); free(W);
        return -1;
    }
    for (int64_t o = 0; o < outer; ++o) {
        for (int64_t i = 0; i < stride; ++i) {
            int64_t base = o * n * stride + i;
            if (bc == ORC_DIRICHLET) {
                /* 0, f_0..f_{n-1}, 0, -f_{n-1}..-f_0 */
                x[0] = 0.0;
                x[n + 1] = 0.0;
                for (int64_t j = 0; j < n; ++j) {
                    x[j + 1] = f[base + j * stride];
                    x[P - 1 - j] = -f[base + j * stride];
                }
            } else if (bc == ORC_NEUMANN) {
                /* f_0..f_{n-1}, f_{n-2}..f_1 */
                for (int64_t j = 0; j < n; ++j) x[j] = f[base + j * stride];
                for (int64_t j = 1; j < n - 1; ++j) x[P - j] = f[base + j * stride];
            } else {
                for (int64_t j = 0; j < n; ++j) x[j] = f[base + j * stride];
            }
            fft_with(x, t, P, W, -1);
            for (int64_t j = 0; j < P; ++j)
                x[j] *= k2_of(j, P, Lp, bc == ORC_PERIODIC ? g->nyquist_zero : 0);
            fft_with(x, t, P, W, +1);
            for (int64_t j = 0; j < n; ++j) {
                int64_t src = bc == ORC_DIRICHLET ? j + 1 : j;
                out[base + j * stride] = creal(x[src]) / (double)P;
            }
        }
    }
    free(x); free(t); free(W);
    return 0;
}

static int64_t n_total(const orc_grid *g)
{
    int64_t t = 1;
    for (int b = 0; b < 3; ++b) t *= (b < g->dims) ? g->n[b] : 1;
    return t;
}

/* out = K src with K = -(hbar/2m*) (d2/dx2 + d2/dy2 + d2/dz2) + V/hbar (Eq. 16),
 * the second derivatives taken spectrally per axis (Eq. 18, one term per axis). */
int orc_apply_K(const double *src, const double *V, double *out, const orc_grid *g)
{
    int64_t nt = n_total(g);
    double *lap = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!lap) return -1;
    double a = g->hbar / (2.0 * g->mass);
    for (int64_t p = 0; p < nt; ++p) out[p] = (V ? V[p] : 0.0) / g->hbar * src[p];
    for (int ax = 0; ax < g->dims; ++ax) {
        if (orc_laplacian_axis(src, lap, g, ax) != 0) {
            free(lap);
            return -1;
        }
        for (int64_t p = 0; p < nt; ++p) out[p] += a * lap[p];
    }
    free(lap);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time stepping (Eq. 14-18).                                                */
/* ------------------------------------------------------------------------ */

/* Advances (psi_R, psi_I) by nsteps steps of the m-stage partitioned
 * symplectic map of Eq. 17: for l = 1..m
 *     psi_R <- psi_R + c_l dt K psi_I        (1 + c_l dt A, Eq. 15/18)
 *     psi_I <- psi_I - d_l dt K psi_R        (1 + d_l dt B, new psi_R)
 * A zero coefficient skips its half-stage.  After every step the value of
 * psi_R + i psi_I at each probe index p is stored at probe_{re,im}[p*nsteps + s]
 * (the time series whose spectrum gives the eigenfrequencies of Tables 2-4). */
int orc_run(double *psiR, double *psiI, const double *V, const orc_grid *g,
            const double *c, const double *d, int m, double dt, int64_t nsteps,
            int n_probe, const int64_t *probe_idx, double *probe_re, double *probe_im)
{
    int64_t nt = n_total(g);
    double *k = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!k) return -1;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int l = 0; l < m; ++l) {
            if (c[l] != 0.0) {
                if (orc_apply_K(psiI, V, k, g)) { free(k); return -1; }
                for (int64_t p = 0; p < nt; ++p) psiR[p] += c[l] * dt * k[p];
            }
            if (d[l] != 0.0) {
                if (orc_apply_K(psiR, V, k, g)) { free(k); return -1; }
                for (int64_t p = 0; p < nt; ++p) psiI[p] -= d[l] * dt * k[p];
            }
        }
        for (int q = 0; q < n_probe; ++q) {
            probe_re[(int64_t)q * nsteps + s] = psiR[probe_idx[q]];
            probe_im[(int64_t)q * nsteps + s] = psiI[probe_idx[q]];
        }
    }
    free(k);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Stability (Eq. 19-30, Table 1).                                           */
/* ------------------------------------------------------------------------ */

/* Per-mode evolution matrix of one full step (Eq. 23) for s = w dt, in the
 * order the stage loop above applies it: M = B_m A_m ... B_1 A_1 with
 * A_l = [[1, c_l s], [0, 1]] and B_l = [[1, 0], [-d_l s, 1]].  Row-major. */
void orc_evolution_matrix(const double *c, const double *d, int m, double s, double *M4)
{
    double a = 1, b = 0, cc = 0, dd = 1; /* [[a, b], [cc, dd]] */
    for (int l = 0; l < m; ++l) {
        /* A_l * M */
        double na = a + c[l] * s * cc, nb = b + c[l] * s * dd;
        a = na; b = nb;
        /* B_l * M */
        double nc = cc - d[l] * s * a, nd = dd - d[l] * s * b;
        cc = nc; dd = nd;
    }
    M4[0] = a; M4[1] = b; M4[2] = cc; M4[3] = dd;
}

double orc_trace(const double *c, const double *d, int m, double s)
{
    double M4[4];
    orc_evolution_matrix(c, d, m, s, M4);
    return M4[0] + M4[3];
}

/* Largest s* such that |tr M(s)| <= 2 for all 0 <= s <= s* (Eq. 25): the first
 * crossing found by a scan in steps of 1e-4, then bisection.  The time step is
 * stable when w_max dt <= s*. */
double orc_stability_limit(const double *c, const double *d, int m)
{
    const double h = 1e-4, smax = 64.0;
    double s = 0.0;
    while (s + h <= smax && fabs(orc_trace(c, d, m, s + h)) <= 2.0) s += h;
    if (s + h > smax) return smax;
    double lo = s, hi = s + h;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (fabs(orc_trace(c, d, m, mid)) <= 2.0) lo = mid;
        else hi = mid;
    }
    return lo;
}

static double theta_of(const double *c, const double *d, int m, double s)
{
    double t = 0.5 * orc_trace(c, d, m, s);
    if (t > 1.0) t = 1.0;
    if (t < -1.0) t = -1.0;
    return acos(t);
}

/* Inverts the numerical dispersion of the map: the mode of K with rate w turns
 * by theta(w dt) = arccos(tr M(w dt)/2) per step (Eq. 24/25: eigenvalues
 * exp(+-i theta) since det M = 1).  Returns s with theta(s) = theta on the
 * first increasing branch of theta (scan in steps of 1e-4, then bisection), so
 * that E = hbar s / dt. */
double orc_phase_correct(double theta, const double *c, const double *d, int m)
{
    const double h = 1e-4;
    double smax = orc_stability_limit(c, d, m);
    double top = 0.0;
    while (top + h <= smax && theta_of(c, d, m, top + h) > theta_of(c, d, m, top)) top += h;
    if (theta >= theta_of(c, d, m, top)) return top;
    double lo = 0.0, hi = top;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (theta_of(c, d, m, mid) < theta) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Eigenfrequencies from a probe time series (Tables 2-4).                   */
/* ------------------------------------------------------------------------ */

/* |sum_n w_n z_n exp(+i theta n)|: the windowed DTFT of the series, which
 * peaks at theta = E dt / hbar for a component z ~ exp(-i E t / hbar). */
static double dtft_abs(const double *re, const double *im, const double *w, int64_t M, double theta)
{
    double sr = 0.0, si = 0.0;
    for (int64_t n = 0; n < M; ++n) {
        double cs = cos(theta * (double)n), sn = sin(theta * (double)n);
        double zr = w[n] * re[n], zi = w[n] * im[n];
        sr += zr * cs - zi * sn;
        si += zr * sn + zi * cs;
    }
    return sqrt(sr * sr + si * si);
}

typedef struct {
    int64_t k;
    double a;
} peak_t;

/* Spectrum analysis of z_n = re[n] + i im[n], n < M (the paper reads the
 * eigenfrequencies off the FFT of the recorded series):
 *  1. symmetric Hann window w_n = (1 - cos(2 pi n/(M-1)))/2 (w = 1 if M = 1);
 *  2. zero pad to nfft and take S_k = |sum_n w_n z_n exp(+2 pi i kn/nfft)|;
 *  3. peaks among 1 <= k < nfft/2 - 1 (positive energies only): S_k is the
 *     largest value within the Hann main-lobe half width h = ceil(2 nfft/M)
 *     bins (S_k > S_j for k-h <= j < k, S_k >= S_j for k < j <= k+h, indices
 *     clipped to [0, nfft/2]), which rejects the window's side lobes, and
 *     S_k >= thresh * max S;
 *  4. the max_peaks largest (ties: lower k first);
 *  5. each refined by 60 golden-section steps maximising the windowed DTFT on
 *     [theta_{k-1}, theta_{k+1}];
 *  6. theta, E = hbar theta / dt and amp = DTFT / sum w, sorted by E.
 * Returns the number of peaks, or -1 on bad input. */
int orc_spectrum(const double *re, const double *im, int64_t M, int64_t nfft, int max_peaks,
                 double thresh, double dt, double hbar, double *theta, double *E, double *amp)
{
    if (M <= 0 || nfft < M || nfft < 4 || max_peaks <= 0) return -1;
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    double *br = (double *)calloc((size_t)nfft, sizeof(double));
    double *bi = (double *)calloc((size_t)nfft, sizeof(double));
    peak_t *pk = (peak_t *)malloc(sizeof(peak_t) * (size_t)(nfft / 2));
    if (!w || !br || !bi || !pk) {
        free(w); free(br); free(bi); free(pk);
        return -1;
    }
    double wsum = 0.0;
    for (int64_t n = 0; n < M; ++n) {
        w[n] = (M == 1) ? 1.0 : 0.5 * (1.0 - cos(TWO_PI * (double)n / (double)(M - 1)));
        wsum += w[n];
        br[n] = w[n] * re[n];
        bi[n] = w[n] * im[n];
    }
    orc_fft(br, bi, nfft, +1);
    double smax = 0.0;
    for (int64_t k = 1; k < nfft / 2; ++k) {
        double s = hypot(br[k], bi[k]);
        if (s > smax) smax = s;
    }
    int np = 0;
    int64_t h = (2 * nfft + M - 1) / M;
    for (int64_t k = 1; k < nfft / 2 - 1; ++k) {
        double s1 = hypot(br[k], bi[k]);
        if (s1 < thresh * smax) continue;
        int is_peak = 1;
        for (int64_t j = k - h; j <= k + h && is_peak; ++j) {
            if (j < 0 || j > nfft / 2 || j == k) continue;
            double sj = hypot(br[j], bi[j]);
            if ((j < k && sj >= s1) || (j > k && sj > s1)) is_peak = 0;
        }
        if (is_peak) {
            pk[np].k = k;
            pk[np].a = s1;
            ++np;
        }
    }
    /* stable insertion sort: amplitude descending, index ascending on ties */
    for (int i = 1; i < np; ++i) {
        peak_t v = pk[i];
        int j = i - 1;
        while (j >= 0 && pk[j].a < v.a) {
            pk[j + 1] = pk[j];
            --j;
        }
        pk[j + 1] = v;
    }
    if (np > max_peaks) np = max_peaks;
    const double g = 0.61803398874989484820; /* (sqrt 5 - 1)/2 */
    for (int i = 0; i < np; ++i) {
        double a = TWO_PI * (double)(pk[i].k - 1) / (double)nfft;
        double b = TWO_PI * (double)(pk[i].k + 1) / (double)nfft;
        double x1 = b - g * (b - a), x2 = a + g * (b - a);
        double f1 = dtft_abs(re, im, w, M, x1), f2 = dtft_abs(re, im, w, M, x2);
        for (int it = 0; it < 60; ++it) {
            if (f1 > f2) {
                b = x2; x2 = x1; f2 = f1;
                x1 = b - g * (b - a);
                f1 = dtft_abs(re, im, w, M, x1);
            } else {
                a = x1; x1 = x2; f1 = f2;
                x2 = a + g * (b - a);
                f2 = dtft_abs(re, im, w, M, x2);
            }
        }
        double t = 0.5 * (a + b);
        theta[i] = t;
        E[i] = hbar * t / dt;
        amp[i] = dtft_abs(re, im, w, M, t) / wsum;
    }
    /* sort the refined peaks by energy */
    for (int i = 1; i < np; ++i) {
        double tv = theta[i], ev = E[i], av = amp[i];
        int j = i - 1;
        while (j >= 0 && E[j] > ev) {
            theta[j + 1] = theta[j]; E[j + 1] = E[j]; amp[j + 1] = amp[j];
            --j;
        }
        theta[j + 1] = tv; E[j + 1] = ev; amp[j + 1] = av;
    }
    free(w); free(br); free(bi); free(pk);
    return np;
}

/* ------------------------------------------------------------------------ */
/* Norm and energy (the integrated |psi|^2 of Fig. 3 and <psi|H|psi>).       */
/* ------------------------------------------------------------------------ */

/* norm = dV sum (psi_R^2 + psi_I^2); energy = dV sum (psi_R H psi_R +
 * psi_I H psi_I) with H = hbar K the Hamiltonian of Eq. 1.  dV is the grid
 * spacing product (L/n periodic, L/(n+1) Dirichlet, L/(n-1) Neumann). */
int orc_norm_energy(const double *psiR, const double *psiI, const double *V,
                    const orc_grid *g, double *norm, double *energy)
{
    int64_t nt = n_total(g);
    double dV = 1.0;
    for (int b = 0; b < g->dims; ++b) {
        int64_t cells = g->bc[b] == ORC_DIRICHLET ? g->n[b] + 1 : g->bc[b] == ORC_NEUMANN ? g->n[b] - 1 : g->n[b];
        dV *= (g->hi[b] - g->lo[b]) / (double)cells;
    }
    double *h = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!h) return -1;
    double sn = 0.0, se = 0.0;
    for (int64_t p = 0; p < nt; ++p) sn += psiR[p] * psiR[p] + psiI[p] * psiI[p];
    if (orc_apply_K(psiR, V, h, g)) { free(h); return -1; }
    for (int64_t p = 0; p < nt; ++p) se += psiR[p] * g->hbar * h[p];
    if (orc_apply_K(psiI, V, h, g)) { free(h); return -1; }
    for (int64_t p = 0; p < nt; ++p) se += psiI[p] * g->hbar * h[p];
    free(h);
    *norm = dV * sn;
    *energy = dV * se;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eigenstates (Figs. 1, 2, 4: the eigenstate belonging to a spectral peak).  */
/* ------------------------------------------------------------------------ */

/* Advances the state by nsteps steps (as orc_run) and accumulates, for each
 * target energy E_k, the windowed Fourier component of the field at every
 * point: acc_k = sum_n w_n psi^n exp(+i E_k t_n / hbar), t_n = (n+1) dt the
 * time after step n, w_n the symmetric Hann window over the nsteps samples
 * (w = 1 if nsteps = 1).  A component exp(-i E t/hbar) of the evolution is
 * kept where E = E_k and suppressed elsewhere by the window, so acc_k is the
 * eigenstate at E_k up to normalisation and phase.  acc arrays: [n_target][n_total]. */
int orc_run_eigen(double *psiR, double *psiI, const double *V, const orc_grid *g,
                  const double *c, const double *d, int m, double dt, int64_t nsteps,
                  int n_target, const double *E, double *acc_re, double *acc_im)
{
    int64_t nt = n_total(g);
    for (int64_t p = 0; p < (int64_t)n_target * nt; ++p) acc_re[p] = acc_im[p] = 0.0;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (orc_run(psiR, psiI, V, g, c, d, m, dt, 1, 0, NULL, NULL, NULL)) return -1;
        double w = (nsteps == 1) ? 1.0 : 0.5 * (1.0 - cos(TWO_PI * (double)s / (double)(nsteps - 1)));
        for (int k = 0; k < n_target; ++k) {
            double ph = E[k] * (double)(s + 1) * dt / g->hbar;
            double cr = w * cos(ph), ci = w * sin(ph);
            for (int64_t p = 0; p < nt; ++p) {
                /* (psiR + i psiI)(cr + i ci) */
                acc_re[(int64_t)k * nt + p] += psiR[p] * cr - psiI[p] * ci;
                acc_im[(int64_t)k * nt + p] += psiR[p] * ci + psiI[p] * cr;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The non-symplectic comparison scheme of Fig. 3: classical Runge-Kutta.     */
/* ------------------------------------------------------------------------ */

/* Classical fourth-order Runge-Kutta for d(psi_R, psi_I)/dt = (K psi_I,
 * -K psi_R) (Eq. 3/4 with K of Eq. 16): k1 = f(y), k2 = f(y + dt/2 k1),
 * k3 = f(y + dt/2 k2), k4 = f(y + dt k3), y += dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * Probes as orc_run. */
int orc_run_rk4(double *psiR, double *psiI, const double *V, const orc_grid *g, double dt, int64_t nsteps,
                int n_probe, const int64_t *probe_idx, double *probe_re, double *probe_im)
{
    int64_t nt = n_total(g);
    double *tr = (double *)malloc(sizeof(double) * (size_t)nt);
    double *ti = (double *)malloc(sizeof(double) * (size_t)nt);
    double *kr = (double *)malloc(sizeof(double) * (size_t)nt);
    double *ki = (double *)malloc(sizeof(double) * (size_t)nt);
    double *ar = (double *)malloc(sizeof(double) * (size_t)nt);
    double *ai = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!tr || !ti || !kr || !ki || !ar || !ai) {
        free(tr); free(ti); free(kr); free(ki); free(ar); free(ai);
        return -1;
    }
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double a[4] = {0.0, 0.5, 0.5, 1.0};
    int rc = 0;
    for (int64_t s = 0; s < nsteps && !rc; ++s) {
        for (int64_t p = 0; p < nt; ++p) {
            tr[p] = ar[p] = psiR[p];
            ti[p] = ai[p] = psiI[p];
        }
        for (int j = 0; j < 4 && !rc; ++j) {
            /* k = f(t): (K t_I, -K t_R) */
            rc |= orc_apply_K(ti, V, kr, g);
            rc |= orc_apply_K(tr, V, ki, g);
            for (int64_t p = 0; p < nt; ++p) {
                ki[p] = -ki[p];
                ar[p] += b[j] * dt * kr[p];
                ai[p] += b[j] * dt * ki[p];
                if (j < 3) {
                    tr[p] = psiR[p] + a[j + 1] * dt * kr[p];
                    ti[p] = psiI[p] + a[j + 1] * dt * ki[p];
                }
            }
        }
        for (int64_t p = 0; p < nt; ++p) {
            psiR[p] = ar[p];
            psiI[p] = ai[p];
        }
        for (int q = 0; q < n_probe; ++q) {
            probe_re[(int64_t)q * nsteps + s] = psiR[probe_idx[q]];
            probe_im[(int64_t)q * nsteps + s] = psiI[probe_idx[q]];
        }
    }
    free(tr); free(ti); free(kr); free(ki); free(ar); free(ai);
    return rc ? -1 : 0;
}
