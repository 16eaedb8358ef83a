// spectra.cuh — single-scattering spectrum model and peak extraction
// (arXiv:2012.00963 Section III.B-C, Eq. 22-35): launchers used by api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "pdv.h"

namespace pdv {

constexpr int kPeakMaxBins = 8192;
constexpr int kPeakNewton = 8;          // Newton steps on the smoothed derivative
constexpr int kPeakThreads = 256;

// Bytes of the per-set constant record the model kernels share.
size_t ss_const_bytes();

// Per-set FP64 constants (one thread per set); invalid sets are counted in
// *d_bad and produce NaN bins.
cudaError_t launch_ss_const(const pdv_ss_set* d_sets, int n_sets, int n_bins, double v_lo,
                            double v_hi, int per_dv, void* d_const, int* d_bad,
                            cudaStream_t st);

// Bin integrals of every set, out[set * n_bins + bin].
cudaError_t launch_ss_bins(const void* d_const, int n_sets, int n_bins, double* d_out,
                           cudaStream_t st);

// cos / sin (2 pi m / n), m = 0..n-1, FP64 rounded to FP32.
cudaError_t launch_twiddles(int n, float2* d_tw, cudaStream_t st);

size_t peak_smem(int n, int k_c);
cudaError_t peak_occupancy(int n, int k_c, int* blocks_per_sm);

// Main-peak extraction of n_spec spectra; bins j_lo..j_hi form the window.
cudaError_t launch_extract(const double* d_spec, int n_spec, int n, int k_c, int j_lo, int j_hi,
                           double v_lo, double dv, double v_fs, const float2* d_tw,
                           pdv_peak* d_out, int grid, cudaStream_t st);

}  // namespace pdv
