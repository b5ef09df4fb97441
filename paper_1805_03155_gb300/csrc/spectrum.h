// spectrum.h -- host interface of the FP64 probe-spectrum kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace spstd {

constexpr int kMaxSpectrumPeaks = 64;

struct SpectrumArgs {
    const double2 *ring;  // [n_probe][cap] samples (psi_R, psi_I)
    int n_probe;
    int p;                // probe, or -1 for the sum of all probes
    int64_t cap;
    int64_t first_slot;   // ring slot of the oldest sample used
    int64_t M;            // samples used (time order from first_slot)
    int64_t nfft;         // power of two, M <= nfft <= max_nfft
    int64_t max_nfft;
    int max_peaks;        // 1..kMaxSpectrumPeaks
    double thresh;
    void *scratch;        // spectrum_scratch_bytes(max_nfft, cap) device bytes
    int *h_npeaks;        // host outputs (written, then the stream is synchronised)
    double *h_theta;
    double *h_amp;
};

size_t spectrum_scratch_bytes(int64_t max_nfft, int64_t cap);
cudaError_t launch_spectrum(const SpectrumArgs &a, cudaStream_t s);
int spectrum_launches(int64_t nfft);

}  // namespace spstd
