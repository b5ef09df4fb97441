// longline.cuh -- the spectral Laplacian (Eq. 7-10) along x lines longer than
// one block can transform on chip, by a four-step FFT through a scratch array.
//
// With N = N1 N2, point n = n1 N2 + n2 and frequency k = k1 + N1 k2:
//   F[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1} sum_n1 z[n1 N2 + n2] W_N1^{n1 k1}.
// The line is a [N1][N2] matrix (rows contiguous).  Three kernels per axis
// application, each on a pair of real lines packed as one complex line:
//   lcol_fwd   length-N1 FFTs down the N2 columns           z   -> C[k1][n2]
//   lrow       per row k1: twiddle W_N^{n2 k1}, length-N2 FFT, multiply by
//              a k^2/N at k = k1 + N1 k2, inverse FFT, conjugate twiddle
//                                                            C   -> C (in place)
//   lcol_inv   inverse length-N1 FFTs down the columns, then
//              dst += result + bV V src (the x axis carries the V term)
// The spectrum is never put back in natural order: the inverse retraces the
// forward steps, so no global transpose is needed.
#pragma once

#include "kernels.cuh"

namespace spstd {

template <typename T>
struct LongArgs {
    const T *src;
    T *dst;
    const T *V;
    cpx<T> *C;           // scratch, n_pairs lines of N complex values, row k1 at k1 N2
    const cpx<T> *tw1;   // W_N1[k], k < N1
    const cpx<T> *tw2;   // W_N2[k], k < N2
    const cpx<T> *twl;   // W_N[k], k < N2: W_N^j = tw1[j / N2] twl[j % N2] for j < N
    T scale;             // a (2 pi/L)^2/N: the multiplier at wrapped index w is scale w^2
    T bV;
    int nyquist_zero;
    int N1, N2;
    int64_t n_rows;      // real lines of N points
    int64_t n_pairs;     // (n_rows + 1)/2
};

// Threads along a column line and columns per block of the column kernels
// (256 threads, LPC N1 = 256 E).
template <typename T, int N1>
__host__ __device__ constexpr int lcol_tt() { return N1 / line_e<T, N1>::value; }
template <typename T, int N1>
__host__ __device__ constexpr int lcol_lpc() { return lcol_tt<T, N1>() >= 256 ? 1 : 256 / lcol_tt<T, N1>(); }
template <typename T, int N1>
__host__ __device__ constexpr size_t lcol_smem()
{
    constexpr int E = line_e<T, N1>::value;
    return align16(sizeof(cpx<T>) * N1) +
           (plan_stages(N1, E) > 1 ? 2 * (size_t)lcol_lpc<T, N1>() * N1 * sizeof(cpx<T>) : 0);
}
template <typename T, int N2>
__host__ __device__ constexpr int lrow_tt() { return N2 / line_e<T, N2>::value; }
template <typename T, int N2>
__host__ __device__ constexpr int lrow_lpc() { return lrow_tt<T, N2>() >= 256 ? 1 : 256 / lrow_tt<T, N2>(); }
// The row kernel keeps its twiddle table in shared memory up to kMaxStagedN
// points; above that it reads the table through L1.  (Staging 4096 FP32
// twiddles, 32 KB, was measured slower: 155 against 114 us per row launch at
// 65536-point lines.)
template <typename T, int N2>
__host__ __device__ constexpr bool lrow_staged() { return N2 <= kMaxStagedN; }
template <typename T, int N2>
__host__ __device__ constexpr size_t lrow_smem()
{
    return (lrow_staged<T, N2>() ? align16(sizeof(cpx<T>) * N2) : 0) +
           2 * (size_t)lrow_lpc<T, N2>() * (N2 + N2 / 32) * sizeof(cpx<T>);
}

// W_N^j for 0 <= j < N (N <= 2^22) from the two tables (one complex
// product); N2 is a power of two, so the split of j is a shift and a mask.
template <typename T, int N2>
__device__ __forceinline__ cpx<T> long_twiddle(const LongArgs<T> &a, uint32_t j)
{
    return cmul<T>(__ldg(a.tw1 + j / N2), __ldg(a.twl + j % N2));
}

// Column tile of block b: pair p, first column n2.
template <int LPC>
__device__ __forceinline__ void lcol_tile(int N2, int64_t b, int64_t *p, int *n2)
{
    const int per = N2 / LPC;
    *p = b / per;
    *n2 = (int)(b - *p * per) * LPC;
}

template <typename T, int N1>
__global__ void __launch_bounds__(lcol_tt<T, N1>() * lcol_lpc<T, N1>())
lcol_fwd_kernel(const LongArgs<T> a)
{
    constexpr int E = line_e<T, N1>::value;
    constexpr int TT = lcol_tt<T, N1>();
    constexpr int LPC = lcol_lpc<T, N1>();
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + align16(sizeof(cpx<T>) * N1));
    const int x = threadIdx.x, t = threadIdx.y;
    for (int i = t * LPC + x; i < N1; i += TT * LPC) s_tw[i] = a.tw1[i];
    __syncthreads();

    int64_t p;
    int n2;
    lcol_tile<LPC>(a.N2, blockIdx.x, &p, &n2);
    n2 += x;
    const int64_t N = (int64_t)N1 * a.N2;
    const bool ok1 = 2 * p + 1 < a.n_rows;
    const T *s0 = a.src + 2 * p * N + n2;
    const T *s1 = s0 + N;
    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t o = (int64_t)(t + e * TT) * a.N2;
        v[e] = mk<T>(s0[o], ok1 ? s1[o] : T(0));
    }
    XcCol<T, LPC> xc{s_ex + x, LPC * N1, 0};
    fft_line<T, N1, E, false>(v, t, xc, s_tw);
    cpx<T> *c = a.C + p * N + n2;
#pragma unroll
    for (int e = 0; e < E; ++e) c[(int64_t)(t + e * TT) * a.N2] = v[e];
}

// FP32: two blocks per SM.  At one (201 registers a thread for N2 = 4096) the
// row kernel ran with 8 warps per SM and was bound by latency; FP64 lines
// (512 threads a block) keep one block, two would spill heavily.
template <typename T>
__host__ __device__ constexpr int lrow_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }
template <typename T, int N2>
__global__ void __launch_bounds__(lrow_tt<T, N2>() * lrow_lpc<T, N2>(), lrow_min_blocks<T>())
lrow_kernel(const LongArgs<T> a)
{
    constexpr int E = line_e<T, N2>::value;
    constexpr int TT = lrow_tt<T, N2>();
    constexpr int LPC = lrow_lpc<T, N2>();
    constexpr int LS = N2 + N2 / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr size_t tb = lrow_staged<T, N2>() ? align16(sizeof(cpx<T>) * N2) : 0;
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + tb);
    const int t = threadIdx.x, l = threadIdx.y;
    const cpx<T> *tw = a.tw2;
    if constexpr (lrow_staged<T, N2>()) {
        cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
        for (int i = l * TT + t; i < N2; i += TT * LPC) s_tw[i] = a.tw2[i];
        __syncthreads();
        tw = s_tw;
    }

    const int64_t rows = a.n_pairs * a.N1;
    const int64_t row = (int64_t)blockIdx.x * LPC + l;
    const bool ok = row < rows;
    const int64_t rr = ok ? row : rows - 1;  // a spare line keeps its threads in the barriers
    const int64_t p = rr / a.N1;
    const int k1 = (int)(rr - p * a.N1);
    const int64_t N = (int64_t)a.N1 * N2;
    cpx<T> *c = a.C + p * N + (int64_t)k1 * N2;

    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int n2 = t + e * TT;
        v[e] = cmul<T>(c[n2], long_twiddle<T, N2>(a, (uint32_t)n2 * (uint32_t)k1));
    }
    XcRow<T, (TT > 32)> xc{s_ex + l * LS, LPC * LS, 0, lane_mask(TT * LPC)};
    fft_line<T, N2, E, false>(v, t, xc, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t k = k1 + (int64_t)a.N1 * (t + e * TT);
        const int64_t w = k <= N / 2 ? k : k - N;
        const T wf = (T)w;
        const T m = (a.nyquist_zero && k == N / 2) ? T(0) : a.scale * (wf * wf);
        v[e].x *= m;
        v[e].y *= m;
    }
    fft_line<T, N2, E, true>(v, t, xc, tw);
    if (ok) {
        // the conjugate twiddles of all elements first, then the products and stores
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc<T>(v[e], long_twiddle<T, N2>(a, (uint32_t)(t + e * TT) * (uint32_t)k1));
#pragma unroll
        for (int e = 0; e < E; ++e) c[t + e * TT] = v[e];
    }
}

template <typename T, int N1>
__global__ void __launch_bounds__(lcol_tt<T, N1>() * lcol_lpc<T, N1>())
lcol_inv_kernel(const LongArgs<T> a)
{
    constexpr int E = line_e<T, N1>::value;
    constexpr int TT = lcol_tt<T, N1>();
    constexpr int LPC = lcol_lpc<T, N1>();
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + align16(sizeof(cpx<T>) * N1));
    const int x = threadIdx.x, t = threadIdx.y;
    for (int i = t * LPC + x; i < N1; i += TT * LPC) s_tw[i] = a.tw1[i];
    __syncthreads();

    int64_t p;
    int n2;
    lcol_tile<LPC>(a.N2, blockIdx.x, &p, &n2);
    n2 += x;
    const int64_t N = (int64_t)N1 * a.N2;
    const cpx<T> *c = a.C + p * N + n2;
    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = c[(int64_t)(t + e * TT) * a.N2];
    XcCol<T, LPC> xc{s_ex + x, LPC * N1, 0};
    fft_line<T, N1, E, true>(v, t, xc, s_tw);

    const bool ok1 = 2 * p + 1 < a.n_rows;
    const int64_t b0 = 2 * p * N + n2;
    // four elements of both lines at a time: their dst, V and src loads are
    // issued together before the stores (dst may alias nothing the compiler
    // can see, so it would otherwise wait on each store)
    constexpr int G = E % 4 == 0 ? 4 : 1;
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += G) {
        T d0[G], d1[G], q0[G], q1[G], s0[G], s1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t o = b0 + (int64_t)(t + (e0 + g) * TT) * a.N2;
            d0[g] = a.dst[o];
            q0[g] = __ldg(a.V + o);
            s0[g] = __ldg(a.src + o);
            d1[g] = ok1 ? a.dst[o + N] : T(0);
            q1[g] = ok1 ? __ldg(a.V + o + N) : T(0);
            s1[g] = ok1 ? __ldg(a.src + o + N) : T(0);
        }
        // the same rounding as one element at a time: dst + result, then + bV V src in one fma
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t o = b0 + (int64_t)(t + (e0 + g) * TT) * a.N2;
            a.dst[o] = fma(a.bV * q0[g], s0[g], d0[g] + v[e0 + g].x);
            if (ok1) a.dst[o + N] = fma(a.bV * q1[g], s1[g], d1[g] + v[e0 + g].y);
        }
    }
}

}  // namespace spstd
