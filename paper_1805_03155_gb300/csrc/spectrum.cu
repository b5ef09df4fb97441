// spectrum.cu -- FP64 eigenfrequency extraction from probe time series
// (Tables 2-4: the eigenfrequencies are read off the Fourier spectrum of the
// field recorded at fixed points while the state evolves).
//
// Steps, all on the device:
//   1. window: z_n = sum of the selected probes' samples in time order,
//      zw_n = w_n z_n with the symmetric Hann window, zero padded to nfft;
//   2. FFT: radix-2 Stockham passes with exp(+2 pi i jk/nfft), giving
//      S(theta_k) = sum_n zw_n exp(+i theta_k n), which peaks at theta =
//      E dt/hbar for a component exp(-i E t/hbar);
//   3. magnitudes |S_k| for k <= nfft/2;
//   4. peak list: the largest |S_k| (one block); then, over the whole grid,
//      a flag for every k in [1, nfft/2 - 1) whose |S_k| is the largest within
//      h = ceil(2 nfft/M) bins (the Hann main-lobe half width, which rejects
//      side lobes) and >= thresh * max; then (one block) the flagged k in
//      order and the max_peaks largest of them, ties to the lower k;
//   5. refinement (one block per peak): 60 golden-section steps maximising
//      |sum_n zw_n exp(+i theta n)| on [theta_{k-1}, theta_{k+1}].
#include <cuda_runtime.h>
#include <stdint.h>

#include "spectrum.h"

namespace spstd {

namespace {

constexpr double kTwoPi = 6.28318530717958647692528676655900577;

__global__ void window_kernel(const double2 *__restrict__ ring, int n_probe, int p, int64_t cap,
                              int64_t first_slot, int64_t M, int64_t nfft, double2 *__restrict__ zw,
                              double2 *__restrict__ buf)
{
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nfft;
         n += (int64_t)gridDim.x * blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (n < M) {
            const int64_t slot = (first_slot + n) % cap;
            if (p >= 0) {
                v = ring[(int64_t)p * cap + slot];
            } else {
                for (int q = 0; q < n_probe; ++q) {
                    const double2 s = ring[(int64_t)q * cap + slot];
                    v.x += s.x;
                    v.y += s.y;
                }
            }
            const double w = (M == 1) ? 1.0 : 0.5 * (1.0 - cospi(2.0 * (double)n / (double)(M - 1)));
            v.x *= w;
            v.y *= w;
            zw[n] = v;
        }
        buf[n] = v;
    }
}

// One radix-2 Stockham pass, span Ns: out[(j/Ns) 2Ns + j%Ns (+Ns)] =
// in[j] +- exp(+i pi (j%Ns)/Ns) in[j + nfft/2].
__global__ void fft2_pass_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int64_t nfft,
                                 int64_t Ns)
{
    const int64_t half = nfft / 2;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < half;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t jm = j % Ns;
        double s, c;
        sincospi((double)jm / (double)Ns, &s, &c);
        const double2 a = in[j];
        const double2 b0 = in[j + half];
        const double2 b = make_double2(b0.x * c - b0.y * s, b0.x * s + b0.y * c);
        const int64_t o = (j / Ns) * 2 * Ns + jm;
        out[o] = make_double2(a.x + b.x, a.y + b.y);
        out[o + Ns] = make_double2(a.x - b.x, a.y - b.y);
    }
}

__global__ void mag_kernel(const double2 *__restrict__ S, int64_t count, double *__restrict__ mag)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        mag[k] = hypot(S[k].x, S[k].y);
}

constexpr int kPeakThreads = 1024;

__device__ __forceinline__ bool better(double a1, int64_t k1, double a2, int64_t k2)
{
    return a1 > a2 || (a1 == a2 && k1 < k2);
}

// The largest |S_k| over 1 <= k < nfft/2 (one block).
__global__ void __launch_bounds__(kPeakThreads)
max_kernel(const double *__restrict__ mag, int64_t nfft, double *__restrict__ smax_out)
{
    __shared__ double s_a[kPeakThreads];
    const int t = threadIdx.x;
    const int64_t half = nfft / 2;
    double mx = 0.0;
    for (int64_t k = 1 + t; k < half; k += kPeakThreads) mx = fmax(mx, mag[k]);
    s_a[t] = mx;
    __syncthreads();
    for (int o = kPeakThreads / 2; o > 0; o >>= 1) {
        if (t < o) s_a[t] = fmax(s_a[t], s_a[t + o]);
        __syncthreads();
    }
    if (t == 0) *smax_out = s_a[0];
}

// flag[k] = 1 where |S_k| >= thresh * max and no bin within h of k beats it
// (ties go to the lower k), for 1 <= k < nfft/2 - 1; 0 elsewhere.
__global__ void flag_kernel(const double *__restrict__ mag, int64_t nfft, int64_t M, double thresh,
                            const double *__restrict__ smax, unsigned char *__restrict__ flag)
{
    const int64_t half = nfft / 2;
    const int64_t h = (2 * nfft + M - 1) / M;
    const double lim = thresh * *smax;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < half;
         k += (int64_t)gridDim.x * blockDim.x) {
        bool pk = k >= 1 && k < half - 1;
        const double s1 = mag[k];
        if (pk && s1 < lim) pk = false;
        for (int64_t j = k - h; pk && j <= k + h; ++j) {
            if (j < 0 || j > half || j == k) continue;
            const double sj = mag[j];
            if ((j < k && sj >= s1) || (j > k && sj > s1)) pk = false;
        }
        flag[k] = pk ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kPeakThreads)
peaks_kernel(const double *__restrict__ mag, const unsigned char *__restrict__ flag, int64_t nfft, int max_peaks,
             int64_t *__restrict__ cand_k, double *__restrict__ cand_a, int64_t *__restrict__ peak_k,
             int *__restrict__ npeaks)
{
    __shared__ double s_a[kPeakThreads];
    __shared__ int64_t s_k[kPeakThreads];
    __shared__ int64_t s_cnt[kPeakThreads];
    const int t = threadIdx.x;
    const int64_t half = nfft / 2;
    // candidates, compacted in k order: contiguous chunk per thread
    const int64_t k_lo = 1, k_hi = half - 1;  // k in [k_lo, k_hi)
    const int64_t span = k_hi > k_lo ? k_hi - k_lo : 0;
    const int64_t chunk = (span + kPeakThreads - 1) / kPeakThreads;
    const int64_t c_lo = k_lo + (int64_t)t * chunk;
    const int64_t c_hi = (c_lo + chunk < k_hi) ? c_lo + chunk : k_hi;
    auto is_peak = [&](int64_t k) -> bool { return flag[k] != 0; };
    int64_t cnt = 0;
    for (int64_t k = c_lo; k < c_hi; ++k) cnt += is_peak(k) ? 1 : 0;
    s_cnt[t] = cnt;
    __syncthreads();
    // exclusive scan (Hillis-Steele on inclusive, then shift)
    for (int o = 1; o < kPeakThreads; o <<= 1) {
        int64_t v = (t >= o) ? s_cnt[t - o] : 0;
        __syncthreads();
        s_cnt[t] += v;
        __syncthreads();
    }
    const int64_t total = s_cnt[kPeakThreads - 1];
    int64_t w = s_cnt[t] - cnt;
    for (int64_t k = c_lo; k < c_hi; ++k) {
        if (is_peak(k)) {
            cand_k[w] = k;
            cand_a[w] = mag[k];
            ++w;
        }
    }
    __syncthreads();
    // 3. the max_peaks best candidates (amplitude descending, k ascending)
    int found = 0;
    for (int i = 0; i < max_peaks; ++i) {
        double ba = -1.0;
        int64_t bk = -1, bi = -1;
        for (int64_t c = t; c < total; c += kPeakThreads) {
            const double a = cand_a[c];
            if (a >= 0.0 && (bk < 0 || better(a, cand_k[c], ba, bk))) {
                ba = a;
                bk = cand_k[c];
                bi = c;
            }
        }
        s_a[t] = ba;
        s_k[t] = bk;
        s_cnt[t] = bi;
        __syncthreads();
        for (int o = kPeakThreads / 2; o > 0; o >>= 1) {
            if (t < o) {
                const bool take = s_k[t + o] >= 0 && (s_k[t] < 0 || better(s_a[t + o], s_k[t + o], s_a[t], s_k[t]));
                if (take) {
                    s_a[t] = s_a[t + o];
                    s_k[t] = s_k[t + o];
                    s_cnt[t] = s_cnt[t + o];
                }
            }
            __syncthreads();
        }
        const int64_t win = s_cnt[0];
        const int64_t wk = s_k[0];
        __syncthreads();
        if (wk < 0) break;
        if (t == 0) {
            peak_k[i] = wk;
            cand_a[win] = -1.0;
        }
        ++found;
        __syncthreads();
    }
    if (t == 0) *npeaks = found;
}

constexpr int kRefineThreads = 256;

// |sum_n zw_n exp(+i theta n)| over the block.  Thread t takes n = t + j T
// (T threads): its phase exp(i theta n) starts from one sincos and advances by
// a complex multiply with exp(i theta T) per sample, so a 50 000-sample series
// costs two sincos per thread instead of one per sample; the recurrence's
// relative rounding stays near (M/T) eps, far below what the golden-section
// search resolves (the square root of the noise of |S| near its maximum).
__device__ double dtft_abs(const double2 *__restrict__ zw, int64_t M, double theta, double *s_re, double *s_im)
{
    double re = 0.0, im = 0.0;
    if ((int64_t)threadIdx.x < M) {
        double s, c, ws, wc;
        sincos(theta * (double)threadIdx.x, &s, &c);
        sincos(theta * (double)kRefineThreads, &ws, &wc);
        for (int64_t n = threadIdx.x; n < M; n += kRefineThreads) {
            const double2 z = zw[n];
            re += z.x * c - z.y * s;
            im += z.x * s + z.y * c;
            const double c2 = c * wc - s * ws;
            s = fma(c, ws, s * wc);
            c = c2;
        }
    }
    s_re[threadIdx.x] = re;
    s_im[threadIdx.x] = im;
    __syncthreads();
    for (int o = kRefineThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_re[threadIdx.x] += s_re[threadIdx.x + o];
            s_im[threadIdx.x] += s_im[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double r = sqrt(s_re[0] * s_re[0] + s_im[0] * s_im[0]);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRefineThreads)
refine_kernel(const double2 *__restrict__ zw, int64_t M, int64_t nfft, const int64_t *__restrict__ peak_k,
              const int *__restrict__ npeaks, double *__restrict__ theta_out, double *__restrict__ amp_out)
{
    __shared__ double s_re[kRefineThreads];
    __shared__ double s_im[kRefineThreads];
    const int i = blockIdx.x;
    if (i >= *npeaks) return;  // uniform over the block
    const double g = 0.61803398874989484820;
    const int64_t k = peak_k[i];
    double a = kTwoPi * (double)(k - 1) / (double)nfft;
    double b = kTwoPi * (double)(k + 1) / (double)nfft;
    double x1 = b - g * (b - a), x2 = a + g * (b - a);
    double f1 = dtft_abs(zw, M, x1, s_re, s_im);
    double f2 = dtft_abs(zw, M, x2, s_re, s_im);
    for (int it = 0; it < 60; ++it) {
        if (f1 > f2) {
            b = x2;
            x2 = x1;
            f2 = f1;
            x1 = b - g * (b - a);
            f1 = dtft_abs(zw, M, x1, s_re, s_im);
        } else {
            a = x1;
            x1 = x2;
            f1 = f2;
            x2 = a + g * (b - a);
            f2 = dtft_abs(zw, M, x2, s_re, s_im);
        }
    }
    const double th = 0.5 * (a + b);
    const double fa = dtft_abs(zw, M, th, s_re, s_im);
    // window sum
    double ws = 0.0;
    for (int64_t n = threadIdx.x; n < M; n += kRefineThreads)
        ws += (M == 1) ? 1.0 : 0.5 * (1.0 - cospi(2.0 * (double)n / (double)(M - 1)));
    s_re[threadIdx.x] = ws;
    __syncthreads();
    for (int o = kRefineThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_re[threadIdx.x] += s_re[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        theta_out[i] = th;
        amp_out[i] = fa / s_re[0];
    }
}

}  // namespace

size_t spectrum_scratch_bytes(int64_t max_nfft, int64_t cap)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(sizeof(double2) * cap)           // zw
         + 2 * al(sizeof(double2) * max_nfft)  // FFT ping-pong
         + al(sizeof(double) * (max_nfft / 2 + 1))  // magnitudes
         + al(sizeof(int64_t) * (max_nfft / 2))     // candidate k
         + al(sizeof(double) * (max_nfft / 2))      // candidate amplitude
         + al(sizeof(int64_t) * kMaxSpectrumPeaks) + al(sizeof(double) * kMaxSpectrumPeaks) * 2 + al(sizeof(int))
         + al(sizeof(double))              // largest magnitude
         + al(max_nfft / 2);               // peak flags
}

cudaError_t launch_spectrum(const SpectrumArgs &a, cudaStream_t s)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    unsigned char *w = (unsigned char *)a.scratch;
    double2 *zw = (double2 *)w;
    w += al(sizeof(double2) * a.cap);
    double2 *b0 = (double2 *)w;
    w += al(sizeof(double2) * a.max_nfft);
    double2 *b1 = (double2 *)w;
    w += al(sizeof(double2) * a.max_nfft);
    double *mag = (double *)w;
    w += al(sizeof(double) * (a.max_nfft / 2 + 1));
    int64_t *cand_k = (int64_t *)w;
    w += al(sizeof(int64_t) * (a.max_nfft / 2));
    double *cand_a = (double *)w;
    w += al(sizeof(double) * (a.max_nfft / 2));
    int64_t *peak_k = (int64_t *)w;
    w += al(sizeof(int64_t) * kMaxSpectrumPeaks);
    double *theta = (double *)w;
    w += al(sizeof(double) * kMaxSpectrumPeaks);
    double *amp = (double *)w;
    w += al(sizeof(double) * kMaxSpectrumPeaks);
    int *np = (int *)w;
    w += al(sizeof(int));
    double *smax = (double *)w;
    w += al(sizeof(double));
    unsigned char *flag = (unsigned char *)w;

    auto grid = [](int64_t n) {
        int64_t b = (n + 255) / 256;
        return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
    };
    window_kernel<<<grid(a.nfft), 256, 0, s>>>(a.ring, a.n_probe, a.p, a.cap, a.first_slot, a.M, a.nfft, zw, b0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double2 *in = b0, *out = b1;
    for (int64_t Ns = 1; Ns < a.nfft; Ns *= 2) {
        fft2_pass_kernel<<<grid(a.nfft / 2), 256, 0, s>>>(in, out, a.nfft, Ns);
        double2 *t = in;
        in = out;
        out = t;
    }
    mag_kernel<<<grid(a.nfft / 2 + 1), 256, 0, s>>>(in, a.nfft / 2 + 1, mag);
    max_kernel<<<1, kPeakThreads, 0, s>>>(mag, a.nfft, smax);
    flag_kernel<<<grid(a.nfft / 2), 256, 0, s>>>(mag, a.nfft, a.M, a.thresh, smax, flag);
    peaks_kernel<<<1, kPeakThreads, 0, s>>>(mag, flag, a.nfft, a.max_peaks, cand_k, cand_a, peak_k, np);
    refine_kernel<<<a.max_peaks, kRefineThreads, 0, s>>>(zw, a.M, a.nfft, peak_k, np, theta, amp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(a.h_npeaks, np, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(a.h_theta, theta, sizeof(double) * a.max_peaks, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(a.h_amp, amp, sizeof(double) * a.max_peaks, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

int spectrum_launches(int64_t nfft)
{
    int passes = 0;
    for (int64_t Ns = 1; Ns < nfft; Ns *= 2) ++passes;
    return 1 + passes + 5;
}

}  // namespace spstd
