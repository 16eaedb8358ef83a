// spectra.cu — single-scattering spectrum model (Eq. 22-28) and peak-based
// parameter extraction (Eq. 29-35, Section III.C) of arXiv:2012.00963.
//
// Single-scattering spectrum. With f the normalised mass density of Eq. 20 and
// Fbar(v) the mass fraction above v, Eq. 28 reads I = P tau0 f exp(-tau0 Fbar).
// Because dFbar/dv = -f, I is the derivative of G(v) = P exp(-tau0 Fbar(v)), so
// the integral of I over a bin [a, c] of the support is exactly G(c) - G(a).
// The kernel writes that difference in the cancellation-free form
//     G(c) - G(a) = -P G(c) expm1(-tau0 (Fbar(a) - Fbar(c))),
//     Fbar(a) - Fbar(c) = E(a) (1 - exp(-(x_c - x_a))) / N,
// where x = beta (v - v_fs) / v_fs, E = exp(-x) and N normalises the law cut
// at v_max (N = 1 without a cut). Per-set constants are prepared in FP64; the
// per-bin work is FP32 (three exponentials and a few FMAs a bin).
//
// Peak extraction. The binned spectrum is low-passed by its real DFT (modes
// 0..k_c), the largest smoothed value on the bin centres of the window is
// found, and Newton steps on the analytic derivative of the trigonometric
// polynomial refine it; I''/I at the peak gives beta (Eq. 34) and the peak
// position gives tau0 (Eq. 31). One block per spectrum, persistent over the
// batch; the twiddle table cos/sin(2 pi m / n) and the spectrum sit in shared
// memory, and every index (j k mod n) is exact integer arithmetic.
#include <cmath>
#include <cstdint>

#include "spectra.cuh"

namespace pdv {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SsConst {
  float A0, D;          // x at edge e is A0 + D e
  float omD;            // 1 - exp(-D): E(a) - E(c) = E(a) omD for a whole bin
  float T, x_max;       // E(v_max) and x(v_max) (T = 0, x_max = inf without a cut)
  float invN;           // 1 / (1 - T)
  float tau0, P;        // optical thickness and prefactor (/ dv with PDV_PER_DV)
  float dx_first;       // x_c - 0 of the bin holding v_fs
  float xa_last;        // x_a of the bin holding v_max
  float dx_last;        // x_max - xa_last
  int b_fs, b_max;      // first and last bin with support
  int cut;              // law cut at v_max
  int bad;              // invalid set: NaN bins
};

__global__ void k_ss_const(const pdv_ss_set* sets, int n_sets, int n_bins, double v_lo,
                           double v_hi, int per_dv, SsConst* out, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sets) return;
  const pdv_ss_set s = sets[i];
  SsConst c{};
  const bool ok = s.beta > 0.0 && isfinite(s.beta) && s.tau0 >= 0.0 && isfinite(s.tau0) &&
                  s.v_fs > 0.0 && isfinite(s.v_fs) && isfinite(s.prefactor) && !isnan(s.v_max);
  if (!ok) {
    c.bad = 1;
    atomicAdd(bad, 1);
    out[i] = c;
    return;
  }
  const double dv = (v_hi - v_lo) / n_bins;
  const double r = s.beta / s.v_fs;
  c.A0 = (float)(r * (v_lo - s.v_fs));
  c.D = (float)(r * dv);
  c.omD = (float)(-expm1(-r * dv));
  c.cut = (s.v_max > s.v_fs && isfinite(s.v_max)) ? 1 : 0;
  const double x_max = c.cut ? r * (s.v_max - s.v_fs) : INFINITY;
  const double T = c.cut ? exp(-x_max) : 0.0;
  c.T = (float)T;
  c.x_max = (float)x_max;
  c.invN = (float)(c.cut ? 1.0 / -expm1(-x_max) : 1.0);
  c.tau0 = (float)s.tau0;
  c.P = (float)(per_dv ? s.prefactor / dv : s.prefactor);
  // bins holding the ends of the support [v_fs, v_max]
  const double e_fs = (s.v_fs - v_lo) / dv;
  const double e_max = c.cut ? (s.v_max - v_lo) / dv : INFINITY;
  const double bf = floor(e_fs);
  const double bm = ceil(e_max) - 1.0;
  c.b_fs = bf < 0.0 ? -1 : (bf >= n_bins ? n_bins : (int)bf);
  c.b_max = bm >= n_bins ? n_bins : (bm < -1.0 ? -2 : (int)bm);
  // exact x at the upper end of the first bin and the lower end of the last
  const double xc_first = fmin(r * (v_lo + (bf + 1.0) * dv - s.v_fs), x_max);
  const double xa_last = fmax(r * (v_lo + bm * dv - s.v_fs), 0.0);
  c.dx_first = (float)xc_first;
  c.xa_last = (float)xa_last;
  c.dx_last = (float)(x_max - xa_last);
  out[i] = c;
}

__global__ void k_ss_bins(const SsConst* cs, int n_sets, int n_bins, double* out) {
  const long long total = (long long)n_sets * n_bins;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int set = (int)(t / n_bins);
    const int b = (int)(t - (long long)set * n_bins);
    const SsConst c = cs[set];
    float val;
    if (c.bad) {
      val = __int_as_float(0x7fc00000);
    } else if (b < c.b_fs || b > c.b_max || (b < 0)) {
      val = 0.0f;
    } else {
      float xa, dx;
      if (b == c.b_fs && b == c.b_max) {
        xa = 0.0f;
        dx = c.x_max;
      } else if (b == c.b_fs) {
        xa = 0.0f;
        dx = c.dx_first;
      } else if (b == c.b_max && c.cut) {
        xa = c.xa_last;
        dx = c.dx_last;
      } else {
        xa = fmaf(c.D, (float)b, c.A0);
        dx = c.D;
      }
      const float Ea = expf(-xa);
      const float om = (dx == c.D) ? c.omD : -expm1f(-dx);
      const float dE = Ea * om;                      // E(a) - E(c)
      float EcT;                                     // E(c) - T
      if (!c.cut) {
        EcT = Ea - dE;
      } else {
        const float y = c.x_max - (xa + dx);         // x_max - x_c >= 0
        EcT = (y < 1.0f) ? c.T * expm1f(fmaxf(y, 0.0f)) : (Ea - dE) - c.T;
      }
      const float Gc = expf(-c.tau0 * EcT * c.invN);
      val = -c.P * Gc * expm1f(-c.tau0 * dE * c.invN);
    }
    out[t] = (double)val;
  }
}

__global__ void k_twiddles(int n, float2* tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * m / n, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

struct PeakSmem {
  size_t o_tw, o_s, o_ab, o_red, bytes;
};

__host__ __device__ inline PeakSmem peak_layout(int n, int k_c) {
  PeakSmem L;
  L.o_tw = 0;
  L.o_s = L.o_tw + sizeof(float2) * (size_t)n;
  L.o_ab = L.o_s + sizeof(float) * (size_t)((n + 1) & ~1);
  L.o_red = L.o_ab + sizeof(float2) * (size_t)(k_c + 1);
  L.bytes = L.o_red + (sizeof(float) + sizeof(int)) * (kPeakThreads / 32);
  return L;
}

// Value and first two derivatives (bin units, times n) of the smoothed
// spectrum at u = J + d, summed by one warp over the modes.
__device__ __forceinline__ void smooth_eval(const float2* tw, const float2* ab, int n, int k_c,
                                            int J, float d, int lane, float* s0, float* s1,
                                            float* s2) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  const float two_over_n = 2.0f / (float)n;
  for (int k = lane; k <= k_c; k += 32) {
    const int m = (int)(((long long)k * J) % n);
    float sp, cp;
    sincospif(two_over_n * (float)k * d, &sp, &cp);
    const float2 t = tw[m];
    const float c = t.x * cp - t.y * sp;             // cos(2 pi k (J + d) / n)
    const float s = t.y * cp + t.x * sp;             // sin(2 pi k (J + d) / n)
    const float2 q = ab[k];
    const float g = k == 0 ? 1.0f : 2.0f;
    const float w = 3.14159265358979f * two_over_n * (float)k;
    const float e = q.x * c + q.y * s;
    a0 = fmaf(g, e, a0);
    a1 = fmaf(g * w, q.y * c - q.x * s, a1);
    a2 = fmaf(-g * w * w, e, a2);
  }
  for (int o = 16; o; o >>= 1) {
    a0 += __shfl_xor_sync(kFull, a0, o);
    a1 += __shfl_xor_sync(kFull, a1, o);
    a2 += __shfl_xor_sync(kFull, a2, o);
  }
  *s0 = a0;
  *s1 = a1;
  *s2 = a2;
}

__global__ void __launch_bounds__(kPeakThreads) k_extract(const double* spec, int n_spec, int n,
                                                          int k_c, int j_lo, int j_hi,
                                                          double v_lo, double dv, double v_fs,
                                                          const float2* twg, pdv_peak* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PeakSmem L = peak_layout(n, k_c);
  float2* tw = reinterpret_cast<float2*>(smem + L.o_tw);
  float* s = reinterpret_cast<float*>(smem + L.o_s);
  float2* ab = reinterpret_cast<float2*>(smem + L.o_ab);
  float* red_v = reinterpret_cast<float*>(smem + L.o_red);
  int* red_j = reinterpret_cast<int*>(red_v + kPeakThreads / 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
  const float inv_n = 1.0f / (float)n;

  for (int sp = blockIdx.x; sp < n_spec; sp += gridDim.x) {
    __syncthreads();                                  // previous spectrum finished
    const double* src = spec + (size_t)sp * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = (float)src[i];
    __syncthreads();
    // real DFT, modes 0..k_c: a_k = sum s_j cos(2 pi j k / n), b_k = sum s_j sin(...)
    for (int k = warp; k <= k_c; k += nw) {
      float a = 0.f, b = 0.f;
      int m = (int)(((long long)lane * k) % n);
      const int step = (int)((32LL * k) % n);
      for (int j = lane; j < n; j += 32) {
        const float2 t = tw[m];
        const float x = s[j];
        a = fmaf(x, t.x, a);
        b = fmaf(x, t.y, b);
        m += step;
        if (m >= n) m -= n;
      }
      for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
      }
      if (lane == 0) ab[k] = make_float2(a, b);
    }
    __syncthreads();
    // smoothed values on the window's bin centres; first maximum wins
    float best = -INFINITY;
    int bj = 0x7fffffff;
    const float a0 = ab[0].x;
    for (int j = j_lo + (int)threadIdx.x; j <= j_hi; j += blockDim.x) {
      float acc = 0.f;
      int m = 0;
      for (int k = 1; k <= k_c; ++k) {
        m += j;
        if (m >= n) m -= n;
        const float2 t = tw[m];
        const float2 q = ab[k];
        acc = fmaf(q.x, t.x, acc);
        acc = fmaf(q.y, t.y, acc);
      }
      const float val = fmaf(2.0f, acc, a0) * inv_n;
      if (val > best) {
        best = val;
        bj = j;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const float ov = __shfl_xor_sync(kFull, best, o);
      const int oj = __shfl_xor_sync(kFull, bj, o);
      if (ov > best || (ov == best && oj < bj)) {
        best = ov;
        bj = oj;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_j[warp] = bj;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? red_v[lane] : -INFINITY;
      bj = lane < nw ? red_j[lane] : 0x7fffffff;
      for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(kFull, best, o);
        const int oj = __shfl_xor_sync(kFull, bj, o);
        if (ov > best || (ov == best && oj < bj)) {
          best = ov;
          bj = oj;
        }
      }
      pdv_peak r;
      r.x_peak = r.i_peak = r.curvature = r.beta = r.tau0 = NAN;
      r.j_max = (j_lo <= j_hi) ? bj : -1;
      r.status = PDV_PEAK_NO_PEAK;
      if (j_lo <= j_hi && best > 0.0f) {
        if (bj == j_lo || bj == j_hi) {
          r.status = PDV_PEAK_EDGE;
        } else {
          float d = 0.f, s0, s1, s2;
          for (int it = 0; it < kPeakNewton; ++it) {
            smooth_eval(tw, ab, n, k_c, bj, d, lane, &s0, &s1, &s2);
            if (!(s2 < 0.0f)) break;
            d = fminf(fmaxf(d - s1 / s2, -1.0f), 1.0f);
          }
          smooth_eval(tw, ab, n, k_c, bj, d, lane, &s0, &s1, &s2);
          const double scale = (v_fs / dv) * (v_fs / dv);
          r.x_peak = (v_lo + ((double)bj + (double)d + 0.5) * dv) / v_fs;
          r.i_peak = (double)s0 * inv_n;
          r.curvature = (double)s2 / (double)s0 * scale;
          if (r.curvature < 0.0) {
            r.status = PDV_PEAK_OK;
            r.beta = sqrt(-r.curvature);
            r.tau0 = exp(r.beta * (r.x_peak - 1.0));
          } else {
            r.status = PDV_PEAK_NOT_MAX;
          }
        }
      }
      if (lane == 0) out[sp] = r;
    }
  }
}

}  // namespace

size_t ss_const_bytes() { return sizeof(SsConst); }

cudaError_t launch_ss_const(const pdv_ss_set* d_sets, int n_sets, int n_bins, double v_lo,
                            double v_hi, int per_dv, void* d_const, int* d_bad,
                            cudaStream_t st) {
  k_ss_const<<<(n_sets + 127) / 128, 128, 0, st>>>(d_sets, n_sets, n_bins, v_lo, v_hi, per_dv,
                                                    static_cast<SsConst*>(d_const), d_bad);
  return cudaGetLastError();
}

cudaError_t launch_ss_bins(const void* d_const, int n_sets, int n_bins, double* d_out,
                           cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long total = (long long)n_sets * n_bins;
  long long blocks = (total + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_ss_bins<<<(int)blocks, 256, 0, st>>>(static_cast<const SsConst*>(d_const), n_sets, n_bins,
                                         d_out);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(int n, float2* d_tw, cudaStream_t st) {
  k_twiddles<<<(n + 255) / 256, 256, 0, st>>>(n, d_tw);
  return cudaGetLastError();
}

size_t peak_smem(int n, int k_c) { return peak_layout(n, k_c).bytes; }

cudaError_t peak_occupancy(int n, int k_c, int* blocks_per_sm) {
  const size_t sm = peak_smem(n, k_c);
  cudaError_t e = cudaFuncSetAttribute(k_extract, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_extract, kPeakThreads,
                                                       sm);
}

cudaError_t launch_extract(const double* d_spec, int n_spec, int n, int k_c, int j_lo, int j_hi,
                           double v_lo, double dv, double v_fs, const float2* d_tw,
                           pdv_peak* d_out, int grid, cudaStream_t st) {
  k_extract<<<grid, kPeakThreads, peak_smem(n, k_c), st>>>(d_spec, n_spec, n, k_c, j_lo, j_hi,
                                                            v_lo, dv, v_fs, d_tw, d_out);
  return cudaGetLastError();
}

}  // namespace pdv
