// kernels.cuh -- the device kernels of one SPSTD half-stage (Eq. 16-18) and
// their helpers.  Each half-stage is
//     dst += a * sum_d L_d src + bV * V * src,
// with L_d = F_d^-1 k_d^2 F_d the spectral -d^2/dx_d^2 along axis d (Eq. 10),
// a = s coef dt hbar/2m* and bV = s coef dt/hbar (s = +1 for psi_R <- psi_I,
// s = -1 for psi_I <- psi_R).  The factor a k^2/N of the inverse transform is
// pre-multiplied into one table per half-stage and axis (FP64 on the host,
// rounded once).
//
// Two real lines travel as the real and imaginary parts of one complex line:
// k^2 is real and even, so F^-1 k^2 F maps a real line to a real line and the
// two never mix.
#pragma once

#include "fft_line.cuh"

namespace spstd {

template <typename T>
struct PassArgs {
    const T *src;
    T *dst;
    const T *V;             // used when use_V != 0
    const cpx<T> *tw;       // W_N[k], k < N
    const T *mult;          // a k^2(n)/N, n < N
    T bV;
    int use_V;
    int64_t n_rows;         // x pass: number of contiguous lines of N points
    int64_t stride;         // strided pass: elements between points along the axis
    int64_t outer_stride;   // strided pass: elements between consecutive line groups
    int64_t n_outer;        // strided pass: number of line groups
    int nx;                 // strided pass: columns (points along x)
    int reverse;            // walk the tiles in reverse order (L2 reuse)
    // x pass of a batch member with a separable potential (FP32): the tables
    // V = vx(x) + vyz(row) whose FP32 sums the V field holds (null: none)
    const T *vx, *vyz;
};

constexpr int kMaxHalfStages = 16;
constexpr int kMaxProbes = 16;

template <typename T>
struct ResidentArgs {
    T *psiR;
    T *psiI;
    const T *V;
    const cpx<T> *tw;
    const T *mult;                // multiplier rows of N values
    T bV[kMaxHalfStages];
    int hfield[kMaxHalfStages];   // 0: psi_R += .. K psi_I ; 1: psi_I += .. K psi_R
    int htable[kMaxHalfStages];   // multiplier row of each executed half-stage
    int nh;
    int64_t nsteps;
    int n_probe;
    int64_t probe_idx[kMaxProbes];
    double2 *ring;
    int64_t cap;
    int64_t *counter;
};

struct ProbeArgs {
    int n_probe;
    int64_t idx[kMaxProbes];
    double2 *ring;
    int64_t cap;
    int64_t *counter;
};

// ---------------------------------------------------------------------------
// Exchange buffers.
// ---------------------------------------------------------------------------

// One contiguous line per thread group, index fastest, one pad slot per 32.
template <typename T, bool BLOCKSYNC>
struct XcRow {
    cpx<T> *base;
    int bufstride;
    int cur;
    unsigned mask;  // lanes of this warp that exist (blocks narrower than a warp)
    __device__ __forceinline__ cpx<T> &at(int idx) { return base[cur * bufstride + idx + (idx >> 5)]; }
    __device__ __forceinline__ void st(int idx, cpx<T> v) { at(idx) = v; }
    __device__ __forceinline__ cpx<T> ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync()
    {
        if constexpr (BLOCKSYNC) __syncthreads();
        else __syncwarp(mask);
    }
    __device__ __forceinline__ void flip() { cur ^= 1; }
};

// LPC column lines side by side, line fastest (conflict-free for a warp that
// spans consecutive lines).
template <typename T, int LPC>
struct XcCol {
    cpx<T> *base;
    int bufstride;
    int cur;
    __device__ __forceinline__ cpx<T> &at(int idx) { return base[cur * bufstride + idx * LPC]; }
    __device__ __forceinline__ void st(int idx, cpx<T> v) { at(idx) = v; }
    __device__ __forceinline__ cpx<T> ld(int idx) { return at(idx); }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    __device__ __forceinline__ void flip() { cur ^= 1; }
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Mask of the lanes of a warp that exist when a block has nthreads threads.
__device__ __forceinline__ unsigned lane_mask(int nthreads)
{
    return nthreads >= 32 ? 0xffffffffu : ((1u << nthreads) - 1u);
}

// Lines up to this length stage their twiddle and multiplier tables in shared
// memory; longer lines read them through L1 (their exchange buffers need the room).
constexpr int kMaxStagedN = 1024;

template <typename T, int N>
__host__ __device__ constexpr size_t table_bytes()
{
    return N <= kMaxStagedN ? align16(sizeof(cpx<T>) * N) + align16(sizeof(T) * N) : 0;
}

template <typename T, int N, int LPC>
__host__ __device__ constexpr size_t xpass_smem()
{
    return table_bytes<T, N>() + 2 * (size_t)LPC * (N + N / 32) * sizeof(cpx<T>);
}
template <typename T, int N, int LPC>
__host__ __device__ constexpr size_t spass_smem()
{
    return table_bytes<T, N>() + 2 * (size_t)LPC * N * sizeof(cpx<T>);
}
template <typename T, int N>
__host__ __device__ constexpr size_t resident_smem()
{
    return align16(sizeof(cpx<T>) * N) + 2 * (size_t)(N + N / 32) * sizeof(cpx<T>);
}

template <typename T, int N>
__device__ __forceinline__ void stage_tables(const PassArgs<T> &a, cpx<T> *s_tw, T *s_mult, int tid,
                                             int nthreads)
{
    for (int i = tid; i < N; i += nthreads) {
        s_tw[i] = a.tw[i];
        s_mult[i] = a.mult[i];
    }
}

// ---------------------------------------------------------------------------
// x pass: contiguous lines.  Block (TT, LPC); line pair lp covers rows 2lp and
// 2lp+1 (the second may be past the end: its half of the complex line is 0).
// ---------------------------------------------------------------------------
// Elements per group of a pass epilogue whose loads are issued together.
__host__ __device__ constexpr int epi_group(int E) { return E % 4 == 0 ? 4 : E % 2 == 0 ? 2 : 1; }

template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__device__ __forceinline__ void xpass_body(const PassArgs<T> &a, int64_t blk)
{
    constexpr int TT = N / E;
    constexpr int LS = N + N / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
    T *s_mult = reinterpret_cast<T *>(smem + align16(sizeof(cpx<T>) * N));
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + table_bytes<T, N>());

    const int t = threadIdx.x;
    const int l = threadIdx.y;
    const cpx<T> *tw = a.tw;
    const T *mult = a.mult;
    if constexpr (N <= kMaxStagedN) {
        stage_tables<T, N>(a, s_tw, s_mult, l * TT + t, TT * LPC);
        __syncthreads();
        tw = s_tw;
        mult = s_mult;
    }

    const int64_t lp = blk * LPC + l;
    const int64_t r0 = 2 * lp, r1 = r0 + 1;
    const bool ok0 = r0 < a.n_rows, ok1 = r1 < a.n_rows;
    const T *s0 = a.src + r0 * N;
    const T *s1 = a.src + r1 * N;

    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + e * TT;
        v[e] = mk<T>(ok0 ? s0[i] : T(0), ok1 ? s1[i] : T(0));
    }
    XcRow<T, (TT > 32)> xc{s_ex + l * LS, LPC * LS, 0, lane_mask(TT * LPC)};
    fft_line<T, N, E, false>(v, t, xc, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const T m = mult[t + e * TT];
        v[e].x *= m;
        v[e].y *= m;
    }
    fft_line<T, N, E, true>(v, t, xc, tw);

    T *d0 = a.dst + r0 * N;
    T *d1 = a.dst + r1 * N;
    const T *V0 = a.use_V ? a.V + r0 * N : nullptr;
    const T *V1 = a.use_V ? a.V + r1 * N : nullptr;
    // G elements of both lines at a time: their dst, V and src loads are issued
    // before the stores (which the compiler may not move loads across)
    constexpr int G = epi_group(E);
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += G) {
        T x0[G], x1[G], q0[G], q1[G], u0[G], u1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int i = t + (e0 + g) * TT;
            x0[g] = ok0 ? d0[i] : T(0);
            x1[g] = ok1 ? d1[i] : T(0);
            q0[g] = ok0 && a.use_V ? V0[i] : T(0);
            q1[g] = ok1 && a.use_V ? V1[i] : T(0);
            u0[g] = ok0 && a.use_V ? s0[i] : T(0);
            u1[g] = ok1 && a.use_V ? s1[i] : T(0);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int i = t + (e0 + g) * TT;
            if (ok0) {
                T acc = x0[g] + v[e0 + g].x;
                if (a.use_V) acc = fma(a.bV * q0[g], u0[g], acc);
                d0[i] = acc;
            }
            if (ok1) {
                T acc = x1[g] + v[e0 + g].y;
                if (a.use_V) acc = fma(a.bV * q1[g], u1[g], acc);
                d1[i] = acc;
            }
        }
    }
}

template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__global__ void __launch_bounds__((N / E) * LPC)
xpass_kernel(const PassArgs<T> a)
{
    xpass_body<T, N, LPC, E>(a, a.reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x);
}

// Batched x pass: members of one shape, tiles_per_member consecutive blocks each.
template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__global__ void __launch_bounds__((N / E) * LPC)
xpass_batch_kernel(const PassArgs<T> *__restrict__ args, int tiles_per_member)
{
    const int member = blockIdx.x / tiles_per_member;
    const PassArgs<T> a = args[member];
    xpass_body<T, N, LPC, E>(a, (int64_t)(blockIdx.x - member * tiles_per_member));
}

// ---------------------------------------------------------------------------
// Strided pass (y or z axis).  Block (LPC, TT): threadIdx.x picks the column
// pair (2p, 2p+1) inside a tile of 2 LPC adjacent x columns, threadIdx.y the
// thread within the line, so each warp reads 2 LPC consecutive values of a
// row per access.  Tile id = outer * n_xt + xt.
// ---------------------------------------------------------------------------
template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__device__ __forceinline__ void spass_body(const PassArgs<T> &a, int64_t blk)
{
    constexpr int TT = N / E;
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
    T *s_mult = reinterpret_cast<T *>(smem + align16(sizeof(cpx<T>) * N));
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + table_bytes<T, N>());

    const int p = threadIdx.x;
    const int t = threadIdx.y;
    stage_tables<T, N>(a, s_tw, s_mult, t * LPC + p, TT * LPC);
    __syncthreads();

    const int n_xt = (a.nx + 2 * LPC - 1) / (2 * LPC);
    const int64_t outer = blk / n_xt;
    const int xt = (int)(blk - outer * n_xt);
    const int c0 = xt * 2 * LPC + 2 * p;
    const bool ok0 = c0 < a.nx, ok1 = c0 + 1 < a.nx;
    const bool vec = ok1 && !(a.nx & 1);
    const int64_t base = outer * a.outer_stride + c0;

    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t off = base + (int64_t)(t + e * TT) * a.stride;
        if (vec) {
            v[e] = *reinterpret_cast<const cpx<T> *>(a.src + off);
        } else {
            v[e] = mk<T>(ok0 ? a.src[off] : T(0), ok1 ? a.src[off + 1] : T(0));
        }
    }
    XcCol<T, LPC> xc{s_ex + p, LPC * N, 0};
    fft_line<T, N, E, false>(v, t, xc, s_tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const T m = s_mult[t + e * TT];
        v[e].x *= m;
        v[e].y *= m;
    }
    fft_line<T, N, E, true>(v, t, xc, s_tw);

    // G elements of the column pair at a time: loads before the stores
    constexpr int G = epi_group(E);
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += G) {
        cpx<T> d[G], w[G], sv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t off = base + (int64_t)(t + (e0 + g) * TT) * a.stride;
            if (vec) {
                d[g] = *reinterpret_cast<const cpx<T> *>(a.dst + off);
                if (a.use_V) {
                    sv[g] = *reinterpret_cast<const cpx<T> *>(a.src + off);
                    w[g] = *reinterpret_cast<const cpx<T> *>(a.V + off);
                }
            } else {
                d[g] = mk<T>(ok0 ? a.dst[off] : T(0), ok1 ? a.dst[off + 1] : T(0));
                if (a.use_V) {
                    sv[g] = mk<T>(ok0 ? a.src[off] : T(0), ok1 ? a.src[off + 1] : T(0));
                    w[g] = mk<T>(ok0 ? a.V[off] : T(0), ok1 ? a.V[off + 1] : T(0));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t off = base + (int64_t)(t + (e0 + g) * TT) * a.stride;
            cpx<T> r = mk<T>(d[g].x + v[e0 + g].x, d[g].y + v[e0 + g].y);
            if (a.use_V) {
                r.x = fma(a.bV * w[g].x, sv[g].x, r.x);
                r.y = fma(a.bV * w[g].y, sv[g].y, r.y);
            }
            if (vec) {
                *reinterpret_cast<cpx<T> *>(a.dst + off) = r;
            } else {
                if (ok0) a.dst[off] = r.x;
                if (ok1) a.dst[off + 1] = r.y;
            }
        }
    }
}

template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__global__ void __launch_bounds__((N / E) * LPC)
spass_kernel(const PassArgs<T> a)
{
    spass_body<T, N, LPC, E>(a, a.reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x);
}

template <typename T, int N, int LPC, int E = line_e<T, N>::value>
__global__ void __launch_bounds__((N / E) * LPC)
spass_batch_kernel(const PassArgs<T> *__restrict__ args, int tiles_per_member)
{
    const int member = blockIdx.x / tiles_per_member;
    const PassArgs<T> a = args[member];
    spass_body<T, N, LPC, E>(a, (int64_t)(blockIdx.x - member * tiles_per_member));
}

// ---------------------------------------------------------------------------
// Resident 1D solver: one block owns a whole 1D grid for all nsteps steps.
// Thread t keeps psi_R, psi_I and V at points t + e TT in registers (the same
// natural layout the line FFT uses), so a half-stage touches global memory
// only for its multiplier table; the probes are written after every step.
// ---------------------------------------------------------------------------
template <typename T, int N>
__device__ __forceinline__ void resident1d_body(const ResidentArgs<T> &a)
{
    constexpr int E = line_e<T, N>::value;
    constexpr int TT = N / E;
    constexpr int LS = N + N / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<T> *s_tw = reinterpret_cast<cpx<T> *>(smem);
    cpx<T> *s_ex = reinterpret_cast<cpx<T> *>(smem + align16(sizeof(cpx<T>) * N));

    const int t = threadIdx.x;
    for (int i = t; i < N; i += TT) s_tw[i] = a.tw[i];

    T R[E], I[E], W[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + e * TT;
        R[e] = a.psiR[i];
        I[e] = a.psiI[i];
        W[e] = a.V[i];
    }
    const int64_t c0 = *a.counter;
    __syncthreads();

    XcRow<T, (TT > 32)> xc{s_ex, LS, 0, lane_mask(TT)};
    for (int64_t step = 0; step < a.nsteps; ++step) {
        for (int h = 0; h < a.nh; ++h) {
            const bool toR = a.hfield[h] == 0;
            const T *mult = a.mult + (int64_t)a.htable[h] * N;
            cpx<T> v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = mk<T>(toR ? I[e] : R[e], T(0));
            fft_line<T, N, E, false>(v, t, xc, s_tw);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const T m = __ldg(mult + t + e * TT);
                v[e].x *= m;
                v[e].y *= m;
            }
            fft_line<T, N, E, true>(v, t, xc, s_tw);
            const T bV = a.bV[h];
            if (toR) {
#pragma unroll
                for (int e = 0; e < E; ++e) R[e] = fma(bV * W[e], I[e], R[e] + v[e].x);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) I[e] = fma(bV * W[e], R[e], I[e] + v[e].x);
            }
        }
        const int64_t slot = (c0 + step) % a.cap;
        for (int q = 0; q < a.n_probe; ++q) {
            const int64_t idx = a.probe_idx[q];
            if ((int)(idx % TT) == t) {
                const int eo = (int)(idx / TT);
                T pr = T(0), pi = T(0);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e == eo) {
                        pr = R[e];
                        pi = I[e];
                    }
                }
                a.ring[(int64_t)q * a.cap + slot] = make_double2((double)pr, (double)pi);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + e * TT;
        a.psiR[i] = R[e];
        a.psiI[i] = I[e];
    }
    __syncthreads();
    if (t == 0) *a.counter = c0 + a.nsteps;
}

template <typename T, int N>
__global__ void __launch_bounds__(N / line_e<T, N>::value)
resident1d_kernel(const ResidentArgs<T> a)
{
    resident1d_body<T, N>(a);
}

// Batched resident solver: block b advances member b (all of length N).
template <typename T, int N>
__global__ void __launch_bounds__(N / line_e<T, N>::value)
resident1d_batch_kernel(const ResidentArgs<T> *__restrict__ args, int64_t nsteps)
{
    ResidentArgs<T> a = args[blockIdx.x];
    a.nsteps = nsteps;
    resident1d_body<T, N>(a);
}

// ---------------------------------------------------------------------------
// Dense line operator (wall boundaries and lengths that are not powers of two):
// along one axis, dst += a * (D src) + bV V src with D the n x n spectral
// second-derivative matrix of that axis (times hbar/2m*), stored transposed
// (entry (i, j) at j n + i) so that consecutive threads read consecutive
// entries.  Line l
// starts at (l / inner) * outer_stride + (l % inner) and steps by stride.
// ---------------------------------------------------------------------------
template <typename T>
struct DenseArgs {
    const T *src;
    T *dst;
    const T *V;      // used when use_V
    const T *D;      // [n][n], transposed: D(i, j) at j * n + i
    T a, bV;
    int use_V;
    int n;
    int64_t stride, inner, outer_stride, n_lines;
};

// Lines per block of the dense pass: the operator column each thread reads
// (one entry per j, coalesced across the block, from L1/L2) serves this many
// lines, whose values sit in shared memory as [n][kDenseLines] (a broadcast
// 16-byte read gives four lines' values).
constexpr int kDenseLines = 16;
constexpr int kDenseMaxThreads = 256;  // one thread per output point (n <= SPSTD_MAX_DENSE_N = 256)

// dst(i, line) += a sum_j D(i, j) src(j, line) (+ bV V src on the x axis) for
// kDenseLines lines per block; thread i accumulates over j in order, so every
// output rounds as a plain per-line loop would.
template <typename T>
__global__ void __launch_bounds__(kDenseMaxThreads) dense_pass_kernel(const DenseArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *X = reinterpret_cast<T *>(smem);  // [n][kDenseLines]
    const int n = a.n;
    const int64_t l0 = (int64_t)blockIdx.x * kDenseLines;
    for (int k = threadIdx.x; k < n * kDenseLines; k += blockDim.x) {
        const int j = k / kDenseLines, c = k % kDenseLines;
        const int64_t l = l0 + c;
        T v = T(0);
        if (l < a.n_lines) v = a.src[(l / a.inner) * a.outer_stride + (l % a.inner) + (int64_t)j * a.stride];
        X[k] = v;
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= n) return;
    T acc[kDenseLines];
#pragma unroll
    for (int c = 0; c < kDenseLines; ++c) acc[c] = T(0);
    for (int j = 0; j < n; ++j) {
        const T d = __ldg(a.D + (int64_t)j * n + i);
        const T *xj = X + j * kDenseLines;
#pragma unroll
        for (int c = 0; c < kDenseLines; ++c) acc[c] = fma(d, xj[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kDenseLines; ++c) {
        const int64_t l = l0 + c;
        if (l >= a.n_lines) break;
        const int64_t off = (l / a.inner) * a.outer_stride + (l % a.inner) + (int64_t)i * a.stride;
        T r = a.dst[off] + a.a * acc[c];
        if (a.use_V) r = fma(a.bV * a.V[off], X[i * kDenseLines + c], r);
        a.dst[off] = r;
    }
}

// Whole 1D grid of n points in one block (thread i owns point i), all steps of
// a call, with the dense operator of the axis: one barrier per half-stage.
template <typename T>
struct DenseResidentArgs {
    T *psiR, *psiI;
    const T *V, *D;
    T a[kMaxHalfStages], bV[kMaxHalfStages];
    int hfield[kMaxHalfStages];
    int nh, n;
    int64_t nsteps;
    int n_probe;
    int64_t probe_idx[kMaxProbes];
    double2 *ring;
    int64_t cap;
    int64_t *counter;
};

template <typename T>
__global__ void dense_resident1d_kernel(const DenseResidentArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *f[2] = {reinterpret_cast<T *>(smem), reinterpret_cast<T *>(smem) + a.n};
    const int i = threadIdx.x;
    const bool own = i < a.n;
    T Vi = T(0);
    if (own) {
        f[0][i] = a.psiR[i];
        f[1][i] = a.psiI[i];
        Vi = a.V[i];
    }
    const int64_t c0 = *a.counter;
    __syncthreads();
    for (int64_t step = 0; step < a.nsteps; ++step) {
        for (int h = 0; h < a.nh; ++h) {
            const int d = a.hfield[h];       // updated field
            const T *src = f[1 - d];
            if (own) {
                T acc = T(0);
                for (int j = 0; j < a.n; ++j) acc = fma(__ldg(a.D + (int64_t)j * a.n + i), src[j], acc);
                f[d][i] = fma(a.bV[h] * Vi, src[i], f[d][i] + a.a[h] * acc);
            }
            __syncthreads();
        }
        const int64_t slot = (c0 + step) % a.cap;
        if (i < a.n_probe) {
            const int64_t idx = a.probe_idx[i];
            a.ring[(int64_t)i * a.cap + slot] = make_double2((double)f[0][idx], (double)f[1][idx]);
        }
        __syncthreads();  // the probes read other threads' points
    }
    if (own) {
        a.psiR[i] = f[0][i];
        a.psiI[i] = f[1][i];
    }
    __syncthreads();
    if (i == 0) *a.counter = c0 + a.nsteps;
}

// ---------------------------------------------------------------------------
// Probe recorder (one block): ring[q][counter % cap] = (psi_R, psi_I)(idx_q).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void probe_kernel(const T *__restrict__ psiR, const T *__restrict__ psiI, const ProbeArgs a)
{
    const int64_t c = *a.counter;
    const int q = threadIdx.x;
    if (q < a.n_probe) {
        const int64_t idx = a.idx[q];
        a.ring[(int64_t)q * a.cap + c % a.cap] = make_double2((double)psiR[idx], (double)psiI[idx]);
    }
    __syncthreads();
    if (q == 0) *a.counter = c + 1;
}

// Probe values at a merged step boundary: the boundary lies inside a merged
// half-stage that updates field `mf` with coefficient c_last + c_first, so the
// recorded value of that field is snap + alpha (now - snap), alpha = c_last /
// (c_last + c_first); the other field is unchanged by it.
template <typename T>
__global__ void probe_snapshot_kernel(const T *__restrict__ psiR, const T *__restrict__ psiI, const ProbeArgs a,
                                      double2 *__restrict__ snap)
{
    const int q = threadIdx.x;
    if (q < a.n_probe) snap[q] = make_double2((double)psiR[a.idx[q]], (double)psiI[a.idx[q]]);
}

template <typename T>
__global__ void probe_merged_kernel(const T *__restrict__ psiR, const T *__restrict__ psiI, const ProbeArgs a,
                                    const double2 *__restrict__ snap, double alpha, int mf)
{
    const int64_t c = *a.counter;
    const int q = threadIdx.x;
    if (q < a.n_probe) {
        const int64_t idx = a.idx[q];
        const double2 s = snap[q];
        double r = (double)psiR[idx], i = (double)psiI[idx];
        if (mf == 0) r = s.x + alpha * (r - s.x);
        else i = s.y + alpha * (i - s.y);
        a.ring[(int64_t)q * a.cap + c % a.cap] = make_double2(r, i);
    }
    __syncthreads();
    if (q == 0) *a.counter = c + 1;
}

// Eigenstate accumulation after a step: acc[k][p] += w_n (psi_R + i psi_I)[p]
// exp(+i theta_k (n + 1)), n = *step (samples taken so far), w_n the Hann
// window over `window` samples; no-op once n >= window.  The last block to
// finish advances *step (completion count in *done, reset for the next step).
template <typename T>
__global__ void eigen_accum_kernel(const T *__restrict__ psiR, const T *__restrict__ psiI,
                                   double2 *__restrict__ acc, int64_t n, int n_target, const double *__restrict__ theta,
                                   int64_t window, int64_t *step, unsigned *done)
{
    __shared__ double2 s_ph[4];
    __shared__ bool s_last;
    const int64_t k = *step;
    if (k < window) {
        if (threadIdx.x < n_target) {
            const double w = window == 1 ? 1.0 : 0.5 * (1.0 - cospi(2.0 * (double)k / (double)(window - 1)));
            double sn, cs;
            sincos(theta[threadIdx.x] * (double)(k + 1), &sn, &cs);
            s_ph[threadIdx.x] = make_double2(w * cs, w * sn);
        }
        __syncthreads();
        for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
            // every target's accumulator is loaded before any is stored, so the
            // loads of a point are in flight together
            double2 a[4];
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < n_target) a[t] = acc[(int64_t)t * n + p];
            if constexpr (sizeof(T) == 4) {
                // FP32 fields: the product in FP32 (the fields carry no more), the
                // running sum in FP64 -- two FP64 adds a target instead of four
                // FP64 products, on a part whose FP64 rate is a small fraction of FP32
                const float zr = psiR[p], zi = psiI[p];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (t < n_target) {
                        const float px = (float)s_ph[t].x, py = (float)s_ph[t].y;
                        a[t].x += (double)fmaf(zr, px, -zi * py);
                        a[t].y += (double)fmaf(zr, py, zi * px);
                        acc[(int64_t)t * n + p] = a[t];
                    }
                }
            } else {
                const double zr = (double)psiR[p], zi = (double)psiI[p];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (t < n_target) {
                        const double2 ph = s_ph[t];
                        a[t].x += zr * ph.x - zi * ph.y;
                        a[t].y += zr * ph.y + zi * ph.x;
                        acc[(int64_t)t * n + p] = a[t];
                    }
                }
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        *done = 0u;
        if (k < window) *step = k + 1;
    }
}

// One Runge-Kutta stage update (Fig. 3's comparison scheme) given hR = H t_I,
// hI = H t_R:  o_R = a_R + cb hR, o_I = a_I - cb hI (the running sum: a = y at
// the first stage, o = y at the last);  and, unless last, the next stage state
// t_R = y_R + ca hR, t_I = y_I - ca hI  (cb, ca = stage weight x dt/hbar).
template <typename T>
__global__ void rk4_update_kernel(const T *yR, const T *yI, const T *__restrict__ hR, const T *__restrict__ hI,
                                  const T *aR, const T *aI, T *oR, T *oI, T *__restrict__ tR, T *__restrict__ tI,
                                  int64_t n, T cb, T ca, int last)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const T r = hR[p], i = hI[p];
        const T ar = aR[p], ai = aI[p];
        if (!last) {
            tR[p] = fma(ca, r, yR[p]);
            tI[p] = fma(-ca, i, yI[p]);
        }
        oR[p] = fma(cb, r, ar);
        oI[p] = fma(-cb, i, ai);
    }
}

// Batched probe recorder: block b records member b.
template <typename T>
struct ProbeMember {
    const T *psiR;
    const T *psiI;
    ProbeArgs p;
};

template <typename T>
__global__ void probe_batch_kernel(const ProbeMember<T> *__restrict__ members)
{
    const ProbeMember<T> &m = members[blockIdx.x];
    const int64_t c = *m.p.counter;
    const int q = threadIdx.x;
    if (q < m.p.n_probe) {
        const int64_t idx = m.p.idx[q];
        m.p.ring[(int64_t)q * m.p.cap + c % m.p.cap] = make_double2((double)m.psiR[idx], (double)m.psiI[idx]);
    }
    __syncthreads();
    if (q == 0) *m.p.counter = c + 1;
}

// ---------------------------------------------------------------------------
// FP64 reductions in a fixed order: partial[b] = sum over block b's grid-stride
// elements of x1 y1 (+ x2 y2), then one block sums the partials.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *s_w)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? s_w[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;  // valid in thread 0
}

template <typename T>
__global__ void dot2_kernel(const T *__restrict__ x1, const T *__restrict__ y1, const T *__restrict__ x2,
                            const T *__restrict__ y2, int64_t n, double *__restrict__ partial)
{
    __shared__ double s_w[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = (double)x1[i] * (double)y1[i];
        if (x2) v = fma((double)x2[i], (double)y2[i], v);
        acc += v;
    }
    acc = block_sum(acc, s_w);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// ---------------------------------------------------------------------------
// Precision conversion of host-staged FP64 data.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void from_f64_kernel(const double *__restrict__ in, T *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}
template <typename T>
__global__ void to_f64_kernel(const T *__restrict__ in, double *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

}  // namespace spstd
