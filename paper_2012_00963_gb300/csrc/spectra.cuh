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

// Bin geometry of an extraction in FP32: x of bin centre 0 (v / v_fs), bin
// width / v_fs, and (v_fs / dv)^2 (curvature from bin units to x units).
struct PeakGeom {
  float x0, dxj, scale;
};

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
                           PeakGeom geom, const float2* d_tw, pdv_peak* d_out, int grid,
                           cudaStream_t st);

// Tiled extraction (64 spectra per block, two register-blocked FP32 products
// with fixed cosine/sine matrices) for cut-offs it covers.
bool peak_tiled(int k_c);
size_t peak_mats_bytes(int n, int k_c, int n_w);
cudaError_t tiled_occupancy(int k_c, int* blocks_per_sm);
cudaError_t launch_extract_tiled(const double* d_spec, int n_spec, int n, int k_c, int j_lo,
                                 int j_hi, PeakGeom geom, const float2* d_tw, float* d_mats,
                                 pdv_peak* d_out,
                                 int blocks_per_sm, int sm_count, cudaStream_t st,
                                 cudaEvent_t e0, cudaEvent_t e1);

// Tensor-core extraction (128 spectra per block; the DFT product on tcgen05
// in split TF32, stage 2 as in the tiled kernel), where its shared memory fits.
bool peak_tc(int k_c, int max_smem);
size_t peak_mats_tc_bytes(int n, int k_c, int n_w);
cudaError_t tc_occupancy(int k_c, int* blocks_per_sm);
cudaError_t launch_extract_tc(const double* d_spec, int n_spec, int n, int k_c, int j_lo, int j_hi,
                              PeakGeom geom, const float2* d_tw, float* d_mats, pdv_peak* d_out,
                              int* d_err, int blocks_per_sm, int sm_count, cudaStream_t st,
                              cudaEvent_t e0, cudaEvent_t e1);

}  // namespace pdv
