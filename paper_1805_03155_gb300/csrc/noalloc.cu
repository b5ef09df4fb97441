// noalloc.cu -- spstd_norm_noalloc: the FP64 norm reduction with its scratch in
// a fixed, file-scope device array instead of caller-provided memory.
//
// It is meant for callers that must not allocate device memory at the point
// of the call: code whose device memory belongs to a framework's pool and may
// not call cudaMalloc behind its back, and hot loops that cannot afford
// cudaMalloc's implicit device-wide synchronisation.  Such a caller passes only
// its inputs and its output; the per-block partial sums go to g_partials below.
//
// g_partials is a host-side stand-in when named from host code, not a device
// address: host code must pass the address cudaGetSymbolAddress returns for the
// current device.  That lookup is done once per device, on the first call made
// with that device current; make that first call before any stream capture.
// The address is cached by device ordinal, which holds for the runtime's
// primary context: a caller on a driver-API context of its own, or after a
// cudaDeviceReset, would get an address from another context.
// Every call on a device shares the one array, which keeps the last call's
// contents: calls that overlap on the GPU race on it and must be serialised
// (for example, issued on one stream).  Nothing needs clearing between calls:
// each call writes every partial slot it reads before it reads it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/spstd.h"
#include "launch.cuh"

using namespace spstd;

namespace {

constexpr int kThreads = 256;
constexpr int kElemsPerBlock = kThreads * 8;  // grid-stride: about 8 elements per thread

// SPSTD_NOALLOC_MAX_PARTIALS doubles (512 KB), held by every GPU that loads the
// library until the process exits.
static __device__ __align__(256) double g_partials[SPSTD_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_addr[kMaxDevices] = {nullptr};

__global__ void scale_kernel(double *v, double s) { *v *= s; }

// Device address of g_partials on the current device (looked up once).
cudaError_t partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t norm_impl(const void *psiR, const void *psiI, int64_t n, double cell_volume, double *d_norm,
                      cudaStream_t s, double *partials, int nblocks)
{
    const T *r = static_cast<const T *>(psiR);
    const T *i = static_cast<const T *>(psiI);
    cudaError_t e = Launch<T>::dot2(r, r, i, i, n, partials, nblocks, s);
    if (e != cudaSuccess) return e;
    e = launch_sum_partials(partials, nblocks, d_norm, s);
    if (e != cudaSuccess) return e;
    scale_kernel<<<1, 1, 0, s>>>(d_norm, cell_volume);
    return cudaGetLastError();
}

}  // namespace

extern "C" spstd_status spstd_norm_noalloc(const void *psiR, const void *psiI, int64_t n, int precision,
                                           double cell_volume, double *d_norm, void *stream)
{
    if (!psiR || !psiI || !d_norm || n <= 0 || (precision != 32 && precision != 64)) return SPSTD_EINVAL;
    const int64_t nblocks = (n + kElemsPerBlock - 1) / kElemsPerBlock;
    if (nblocks > SPSTD_NOALLOC_MAX_PARTIALS) return SPSTD_EINVAL;  // n above SPSTD_NOALLOC_MAX_ELEMS
    double *partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) return SPSTD_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e =
        precision == 32 ? norm_impl<float>(psiR, psiI, n, cell_volume, d_norm, s, partials, (int)nblocks)
                        : norm_impl<double>(psiR, psiI, n, cell_volume, d_norm, s, partials, (int)nblocks);
    return e == cudaSuccess ? SPSTD_OK : SPSTD_ECUDA;
}
