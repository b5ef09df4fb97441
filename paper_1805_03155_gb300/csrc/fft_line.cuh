// fft_line.cuh -- register/shared-memory Stockham FFT of one complex line,
// the building block of every spectral-derivative kernel (Eq. 7-10).
//
// A line of N complex points is held by TT = N/E threads, thread t owning the
// elements t + e*TT (e < E) in registers ("natural layout").  N is a power of
// two, or three times one (then E is a multiple of 3 and the first stage's
// radix carries the factor 3).  The transform is
// a Stockham autosort sequence of radix-R stages (R divides E): stage s with
// span Ns (product of the earlier radices) takes butterfly j's inputs from
// j + r*N/R, multiplies them by W_N^{(j mod Ns) r N/(Ns R)}, applies a radix-R
// DFT and writes output r to (j/Ns) Ns R + (j mod Ns) + r Ns.  With thread t
// running butterflies j = t + q*TT, both the inputs of the first stage and the
// outputs of the last stage are in the natural layout, so a line enters from
// global memory and leaves to it without any reordering, and only the
// boundaries between stages go through shared memory (double buffered, one
// barrier per exchange).
//
// Twiddles come from a table W[k] = exp(-2 pi i k/N) computed in FP64 on the
// host and rounded once to the working precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spstd {

template <typename T> struct cpx_traits;
template <> struct cpx_traits<float> { using type = float2; };
template <> struct cpx_traits<double> { using type = double2; };
template <typename T> using cpx = typename cpx_traits<T>::type;

template <typename T>
__device__ __forceinline__ cpx<T> mk(T x, T y)
{
    cpx<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// a * b
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b)
{
    return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b)
{
    return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// a * (-i) for the forward sign, a * (+i) for the inverse
template <typename T, bool INV>
__device__ __forceinline__ cpx<T> rot90(cpx<T> a)
{
    return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// cos(2 pi k/16), sin(2 pi k/16) for k = 0..7 (the radix-16 twiddles).
__host__ __device__ constexpr double c16(int k)
{
    return k == 0 ? 1.0
         : k == 1 ? 0.92387953251128675613
         : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.38268343236508977173
         : k == 4 ? 0.0
         : k == 5 ? -0.38268343236508977173
         : k == 6 ? -0.70710678118654752440
                  : -0.92387953251128675613;
}
__host__ __device__ constexpr double s16(int k) { return k <= 4 ? c16(4 - k) : c16(k - 4); }

// cos(2 pi k/24) for k = 0..6: 1, (sqrt 6 + sqrt 2)/4, sqrt 3/2, sqrt 2/2, 1/2,
// (sqrt 6 - sqrt 2)/4, 0; the rest of the circle by symmetry.  The twiddles of
// the radix-3, 6, 12 and 24 DFTs are multiples of 2 pi/24.
__host__ __device__ constexpr double c24q(int k)
{
    return k == 0 ? 1.0
         : k == 1 ? 0.96592582628906828675
         : k == 2 ? 0.86602540378443864676
         : k == 3 ? 0.70710678118654752440
         : k == 4 ? 0.5
         : k == 5 ? 0.25881904510252076235
                  : 0.0;
}
__host__ __device__ constexpr double c24(int k)
{
    return k < 0 ? c24(k + 24) : k >= 24 ? c24(k - 24)
         : k <= 6 ? c24q(k) : k <= 12 ? -c24q(12 - k) : k <= 18 ? -c24q(k - 12) : c24q(24 - k);
}
__host__ __device__ constexpr double s24(int k) { return c24(k - 6); }

// v * exp(-+ 2 pi i k/R) with k, R compile-time (R | 16).
template <typename T, bool INV, int R, int K>
__device__ __forceinline__ cpx<T> twc(cpx<T> v)
{
    constexpr int k16 = K * (16 / R);
    if constexpr (k16 == 0) {
        return v;
    } else if constexpr (k16 == 4) {
        return rot90<T, INV>(v);
    } else {
        constexpr T cr = (T)c16(k16);
        constexpr T sr = (T)s16(k16);
        // exp(-i a) = (cos a, -sin a) forward; (cos a, +sin a) inverse
        if constexpr (INV)
            return mk<T>(fma(v.x, cr, -v.y * sr), fma(v.x, sr, v.y * cr));
        else
            return mk<T>(fma(v.x, cr, v.y * sr), fma(v.y, cr, -v.x * sr));
    }
}

// v * exp(-+ 2 pi i k/R) with k, R compile-time (R | 24).
template <typename T, bool INV, int R, int K>
__device__ __forceinline__ cpx<T> twc24(cpx<T> v)
{
    constexpr int k24 = (K * (24 / R)) % 24;
    if constexpr (k24 == 0) {
        return v;
    } else if constexpr (k24 == 6) {
        return rot90<T, INV>(v);
    } else if constexpr (k24 == 12) {
        return mk<T>(-v.x, -v.y);
    } else {
        constexpr T cr = (T)c24(k24);
        constexpr T sr = (T)s24(k24);
        if constexpr (INV)
            return mk<T>(fma(v.x, cr, -v.y * sr), fma(v.x, sr, v.y * cr));
        else
            return mk<T>(fma(v.x, cr, v.y * sr), fma(v.y, cr, -v.x * sr));
    }
}

template <typename T, bool INV, int R, int S = 1>
struct DFT;

// Radix R = 3P (P a power of two, R | 24): decimation in time into three
// interleaved sequences of length P, their DFTs, the twiddles W_R^{r k}, and a
// 3-point DFT for each k:  X[k + P s] = sum_r W_3^{r s} (W_R^{r k} A_r[k]).
template <typename T, bool INV, int R, int S>
struct DFT3 {
    static constexpr int P = R / 3;
    template <int K>
    __device__ __forceinline__ static void combine(cpx<T> *u, cpx<T> *out)
    {
        if constexpr (K < P) {
            // 3-point DFT with W_3 = exp(-+ 2 pi i/3) = -1/2 -+ i sqrt3/2
            const cpx<T> a = u[(3 * K) * S];
            const cpx<T> b = twc24<T, INV, R, K>(u[(3 * K + 1) * S]);
            const cpx<T> c = twc24<T, INV, R, 2 * K>(u[(3 * K + 2) * S]);
            const cpx<T> t1 = cadd<T>(b, c), t2 = csub<T>(b, c);
            constexpr T h = (T)c24q(2);  // sqrt 3 / 2
            const cpx<T> m = mk<T>(fma((T)-0.5, t1.x, a.x), fma((T)-0.5, t1.y, a.y));
            out[K] = cadd<T>(a, t1);
            // forward: X1 = m - i h t2, X2 = m + i h t2 (inverse: the signs swap)
            const cpx<T> iht = mk<T>(-h * t2.y, h * t2.x);  // i h t2
            out[K + P] = INV ? cadd<T>(m, iht) : csub<T>(m, iht);
            out[K + 2 * P] = INV ? csub<T>(m, iht) : cadd<T>(m, iht);
            combine<K + 1>(u, out);
        }
    }
    __device__ __forceinline__ static void run(cpx<T> *u)
    {
        DFT<T, INV, P, 3 * S>::run(u);
        DFT<T, INV, P, 3 * S>::run(u + S);
        DFT<T, INV, P, 3 * S>::run(u + 2 * S);
        cpx<T> out[R];
        combine<0>(u, out);
#pragma unroll
        for (int k = 0; k < R; ++k) u[k * S] = out[k];
    }
};

// In-register radix-R DFT of u[0], u[S], ..., u[(R-1)S] (stride S), in place,
// natural output order.  R in {1, 2, 4, 8, 16} (split radix-2 recursion) or
// R in {3, 6, 12, 24} (DFT3 above).
template <typename T, bool INV, int R, int S>
struct DFT {
    template <int K>
    __device__ __forceinline__ static void combine(cpx<T> *u)
    {
        if constexpr (K < R / 2) {
            // after the two half DFTs: evens at u[0..R/2) (stride 2S), odds at u[S..] (stride 2S)
            cpx<T> e = u[(2 * K) * S];
            cpx<T> o = twc<T, INV, R, K>(u[(2 * K + 1) * S]);
            u[(2 * K) * S] = cadd<T>(e, o);
            u[(2 * K + 1) * S] = csub<T>(e, o);
            combine<K + 1>(u);
        }
    }
    __device__ __forceinline__ static void run(cpx<T> *u)
    {
        if constexpr (R % 3 == 0) {
            DFT3<T, INV, R, S>::run(u);
        } else if constexpr (R == 1) {
            return;
        } else if constexpr (R == 2) {
            cpx<T> a = u[0], b = u[S];
            u[0] = cadd<T>(a, b);
            u[S] = csub<T>(a, b);
        } else {
            // decimation in time: DFT of even-indexed and odd-indexed halves
            DFT<T, INV, R / 2, 2 * S>::run(u);
            DFT<T, INV, R / 2, 2 * S>::run(u + S);
            // X[k] = E[k] + w^k O[k], X[k + R/2] = E[k] - w^k O[k]; the results
            // land interleaved (X[k] at 2k, X[k+R/2] at 2k+1) and are put back in
            // natural order below.
            combine<0>(u);
            cpx<T> tmp[R];
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                tmp[k] = u[(2 * k) * S];
                tmp[k + R / 2] = u[(2 * k + 1) * S];
            }
#pragma unroll
            for (int k = 0; k < R; ++k) u[k * S] = tmp[k];
        }
    }
};

// ---------------------------------------------------------------------------
// Stage plans.  E = elements per thread (a power of two, or 3 times one),
// N = E * TT with TT a power of two.  The first stage has radix min(N, E); the
// rest of N/E is split into as many stages of radix P = the largest power of
// two dividing E as fit, plus one smaller remainder stage placed second.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
__host__ __device__ constexpr int p2div(int x) { return x & -x; }

__host__ __device__ constexpr int plan_stages(int N, int E)
{
    return N <= E ? 1
                  : 1 + ((ilog2c(N / E) % ilog2c(p2div(E))) ? 1 : 0) + ilog2c(N / E) / ilog2c(p2div(E));
}
__host__ __device__ constexpr int plan_radix(int N, int E, int s)
{
    return N <= E ? N
         : s == 0 ? E
         : (s == 1 && (ilog2c(N / E) % ilog2c(p2div(E)))) ? (1 << (ilog2c(N / E) % ilog2c(p2div(E))))
                                                          : p2div(E);
}
__host__ __device__ constexpr int plan_span(int N, int E, int s)
{
    return s == 0 ? 1 : plan_span(N, E, s - 1) * plan_radix(N, E, s - 1);
}

// Exchange buffer concept (XC):
//   st(idx, value)  -- write element idx of this thread's line
//   ld(idx)         -- read element idx of this thread's line
//   sync()          -- barrier over every thread sharing the buffer
//   flip()          -- switch to the other half of the double buffer

template <typename T, int N, int E, bool INV, int S, typename XC>
__device__ __forceinline__ void fft_stage(cpx<T> (&v)[E], const int t, XC &xc,
                                          const cpx<T> *__restrict__ tw)
{
    constexpr int NS = plan_stages(N, E);
    if constexpr (S < NS) {
        constexpr int R = plan_radix(N, E, S);
        constexpr int Ns = plan_span(N, E, S);
        constexpr int TT = N / E;
        constexpr int Q = E / R;
        static_assert(E % R == 0, "stage radix must divide the elements per thread");
        static_assert(N % E == 0 && ((N / E) & (N / E - 1)) == 0, "N/E must be a power of two");
        if constexpr (S > 0) {
            xc.sync();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = xc.ld(t + e * TT);
            xc.flip();
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = t + q * TT;
            cpx<T> u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[q + r * Q];
            const int jm = j % Ns;
            if constexpr (S > 0) {
                constexpr int step = N / (Ns * R);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const cpx<T> w = tw[jm * r * step];
                    u[r] = INV ? cmulc<T>(u[r], w) : cmul<T>(u[r], w);
                }
            }
            DFT<T, INV, R>::run(u);
            if constexpr (S == NS - 1) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[q + r * Q] = u[r];
            } else {
                const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
                for (int r = 0; r < R; ++r) xc.st(base + r * Ns, u[r]);
            }
        }
        fft_stage<T, N, E, INV, S + 1>(v, t, xc, tw);
    }
}

// Unnormalised DFT of the line held in v (natural layout in and out):
// forward exp(-2 pi i jk/N) or inverse exp(+2 pi i jk/N).
template <typename T, int N, int E, bool INV, typename XC>
__device__ __forceinline__ void fft_line(cpx<T> (&v)[E], const int t, XC &xc,
                                         const cpx<T> *__restrict__ tw)
{
    fft_stage<T, N, E, INV, 0>(v, t, xc, tw);
}

// Elements per thread for a line of N points in precision T: 16 FP32 / 8
// FP64 for a power-of-two N; 12 (or N, below that) for N = 3 * 2^k, so that
// the first stage takes the factor 3.
template <typename T> struct max_e;
template <> struct max_e<float> { static constexpr int value = 16; };
template <> struct max_e<double> { static constexpr int value = 8; };
template <typename T, int N>
struct line_e {
    static constexpr int value = N % 3 == 0 ? (N < 12 ? N : 12) : (N < max_e<T>::value ? N : max_e<T>::value);
};

}  // namespace spstd
