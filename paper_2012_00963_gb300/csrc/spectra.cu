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
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "spectra.cuh"

namespace pdv {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// binary64 -> binary32, round to nearest even, in integer operations (the
// FP64 pipe of this GPU is narrow). Results below the smallest normal binary32
// flush to a signed zero; infinities and NaNs pass through.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (unsigned)((b >> 29) & 0x7fffffu) |
                                          ((b & 0xfffffffffffffull) ? 0x400000u : 0u));
  // mantissa with the hidden bit, rounded to 24 bits (a carry may bump the exponent)
  unsigned long long m = (b & 0xfffffffffffffull) >> 0;
  const unsigned long long r = m + 0x0fffffffull + ((m >> 29) & 1ull);
  int e = ex - 1023 + 127 + (int)(r >> 52);
  const unsigned mf = (unsigned)((r >> 29) & 0x7fffffu);
  if (ex == 0 || e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | mf);
}

// binary32 -> binary64 (exact), in integer operations; binary32 subnormals
// flush to a signed zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  if (ex == 0) return __longlong_as_double((long long)sign);
  if (ex == 0xff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | m));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 896u) << 52) | m));
}

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
  // exact x at the edge above v_fs (edge 0 when v_fs < v_lo) and at the edge
  // below v_max (edge n_bins when v_max > v_hi), clamped to the support
  const double ef = (double)c.b_fs + 1.0, em = (double)c.b_max;
  const double xc_first = fmax(fmin(r * (v_lo + ef * dv - s.v_fs), x_max), 0.0);
  const double xa_last = fmax(fmin(r * (v_lo + em * dv - s.v_fs), x_max), 0.0);
  c.dx_first = (float)xc_first;
  c.xa_last = (float)xa_last;
  c.dx_last = (float)(x_max - xa_last);
  out[i] = c;
}

// x at edge e of the bins, clamped to the support [0, x_max]; the two edges
// next to the ends of the support come exactly from the FP64 constants.
__device__ __forceinline__ float ss_edge_x(const SsConst& c, int e) {
  if (e <= c.b_fs) return 0.0f;
  if (e > c.b_max) return c.x_max;
  if (e == c.b_fs + 1) return c.dx_first;
  if (e == c.b_max) return c.xa_last;
  return fmaf(c.D, (float)e, c.A0);
}

// exp(-tau0 Fbar) at an edge, from x_e and E_e = exp(-x_e)
__device__ __forceinline__ float ss_edge_g(const SsConst& c, float x, float E) {
  float EcT = E;                                   // E - T
  if (c.cut) {
    const float y = c.x_max - x;
    EcT = (y < 1.0f) ? c.T * expm1f(fmaxf(y, 0.0f)) : E - c.T;
  }
  return expf(-c.tau0 * EcT * c.invN);
}

// Peak position, value and curvature from the converged Newton state, all in
// FP32: x = x_0 + (J + d) dv / v_fs is formed as (x_0 + J dv/v_fs) + d dv/v_fs
// so the fractional part keeps its precision next to a large J.
__device__ __forceinline__ void peak_finish(pdv_peak& r, int J, float d, float q0, float q2,
                                            float inv_n, const PeakGeom& g) {
  const float x = fmaf(d, g.dxj, fmaf((float)J, g.dxj, g.x0));
  const float curv = q2 / q0 * g.scale;
  r.x_peak = f32_to_f64(x);
  r.i_peak = f32_to_f64(q0 * inv_n);
  r.curvature = f32_to_f64(curv);
  if (curv < 0.0f) {
    const float beta = sqrtf(-curv);
    r.status = PDV_PEAK_OK;
    r.beta = f32_to_f64(beta);
    r.tau0 = f32_to_f64(expf(beta * (x - 1.0f)));
  } else {
    r.status = PDV_PEAK_NOT_MAX;
  }
}

constexpr int kRun = 4;          // consecutive bins per thread (edges shared)

__global__ void k_ss_bins(const SsConst* cs, int n_sets, int n_bins, double* out) {
  const unsigned runs = (unsigned)((n_bins + kRun - 1) / kRun);
  const unsigned long long total = (unsigned long long)n_sets * runs;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       t < total; t += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned set, run;
    if (total <= 0xffffffffull) {
      set = (unsigned)t / runs;
      run = (unsigned)t - set * runs;
    } else {
      set = (unsigned)(t / runs);
      run = (unsigned)(t - (unsigned long long)set * runs);
    }
    const SsConst c = cs[set];
    double* o = out + (size_t)set * n_bins;
    const int b0 = (int)run * kRun;
    if (c.bad) {
      for (int i = 0; i < kRun && b0 + i < n_bins; ++i) o[b0 + i] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    float xa = ss_edge_x(c, b0);
    float Ea = expf(-xa);
#pragma unroll
    for (int i = 0; i < kRun; ++i) {
      const int b = b0 + i;
      if (b >= n_bins) break;
      const float xc = ss_edge_x(c, b + 1);
      float dx, Ec;
      if (b > c.b_fs && b < c.b_max) {             // whole bin inside the support
        dx = c.D;
        Ec = Ea * (1.0f - c.omD);
      } else if (b == c.b_fs && b == c.b_max) {
        dx = c.x_max;
        Ec = expf(-xc);
      } else if (b == c.b_fs) {
        dx = c.dx_first;
        Ec = expf(-xc);
      } else if (b == c.b_max) {
        dx = c.dx_last;
        Ec = expf(-xc);
      } else {                                     // outside the support
        dx = 0.0f;
        Ec = Ea;
      }
      const float om = (dx == c.D) ? c.omD : -expm1f(-dx);
      const float Gc = ss_edge_g(c, xc, Ec);
      const float val = -c.P * Gc * expm1f(-c.tau0 * (Ea * om) * c.invN);
      o[b] = f32_to_f64(val);
      xa = xc;
      Ea = Ec;
    }
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
  int m = (lane * J) % n;                           // (k J) mod n, k = lane + 32 i (< 2^18: 32 bits)
  const int step = (32 * J) % n;
  for (int k = lane; k <= k_c; k += 32, m = (m + step >= n) ? m + step - n : m + step) {
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
                                                          PeakGeom geom, const float2* twg,
                                                          pdv_peak* out) {
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
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = f64_to_f32(src[i]);
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
          // Newton on s' = 0; a step below 1e-6 bin ends it (the values of
          // the last evaluation then stand for the final d)
          smooth_eval(tw, ab, n, k_c, bj, d, lane, &s0, &s1, &s2);
          for (int it = 0; it < kPeakNewton && s2 < 0.0f; ++it) {
            const float nd = fminf(fmaxf(d - s1 / s2, -1.0f), 1.0f);
            const bool done = fabsf(nd - d) <= 1e-6f;
            d = nd;
            if (done) break;
            smooth_eval(tw, ab, n, k_c, bj, d, lane, &s0, &s1, &s2);
          }
          peak_finish(r, bj, d, s0, s2, inv_n, geom);
        }
      }
      if (lane == 0) out[sp] = r;
    }
  }
}

// ------------------------------------------------------------------ tiled extraction
// Batched form of the same computation for cut-offs up to kTileMaxK2 / 2 - 1
// modes. A block takes a tile of kTS spectra. The DFT (modes 0..k_c) of the
// tile is the product of the tile (kTS x n) with the fixed matrix
// F[j][2k] = cos(2 pi j k / n), F[j][2k+1] = sin(2 pi j k / n); the smoothed
// values on the window's bin centres are the product of those coefficients
// with G[2k][j] = g_k cos(2 pi k (j_lo + j) / n) / n, G[2k+1][j] = g_k sin(...) / n
// (g_0 = 1, g_k = 2). F and G are built once per call (FP64 rounded to FP32)
// and stay in L2; each block streams them through shared memory in chunks and
// accumulates a 4 x 6 register tile per thread. The grid maximum and the
// Newton refinement then run per spectrum from the coefficients kept in
// shared memory.
constexpr int kTS = 64;          // spectra per tile
constexpr int kNT = 96;          // output columns per pass (16 threads x 6)
constexpr int kJC = 32;          // reduction chunk
constexpr int kAS = kTS + 4;     // row stride of spectrum-major operands (float4 aligned)
constexpr int kTileMaxK2 = 192;  // padded 2 (k_c + 1) handled by the tiled kernel

__host__ __device__ inline int pad_to(int x, int m) { return (x + m - 1) / m * m; }

struct TileSmem {
  size_t o_a, o_b, o_c, o_red, bytes;
};

__host__ __device__ inline TileSmem tile_layout(int k2p) {
  TileSmem L;
  L.o_a = 0;
  L.o_b = L.o_a + sizeof(float) * kJC * kAS;
  L.o_c = L.o_b + 2 * sizeof(float) * kJC * kNT;           // two buffers
  L.o_red = L.o_c + sizeof(float) * (size_t)k2p * kAS;
  L.bytes = L.o_red + (sizeof(float) + sizeof(int)) * kTS;
  return L;
}

// F: [n_p][k2p] and G: [k2p][nw_p], zero in the padding.
__global__ void k_peak_mats(int n, int k_c, int n_p, int k2p, int j_lo, int n_w, int nw_p,
                            float* F, float* G) {
  const long long nF = (long long)n_p * k2p, nG = (long long)k2p * nw_p;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nF + nG;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nF) {
      const int j = (int)(t / k2p), r = (int)(t % k2p), k = r >> 1;
      float v = 0.0f;
      if (j < n && k <= k_c) {
        double s, c;
        sincospi(2.0 * (double)(((long long)j * k) % n) / n, &s, &c);
        v = (float)((r & 1) ? s : c);
      }
      F[t] = v;
    } else {
      const long long u = t - nF;
      const int r = (int)(u / nw_p), j = (int)(u % nw_p), k = r >> 1;
      float v = 0.0f;
      if (j < n_w && k <= k_c && !(k == 0 && (r & 1))) {
        double s, c;
        sincospi(2.0 * (double)(((long long)(j_lo + j) * k) % n) / n, &s, &c);
        v = (float)(((r & 1) ? s : c) * (k == 0 ? 1.0 : 2.0) / n);
      }
      G[u] = v;
    }
  }
}

// acc[4][6] += A[rows ty*4..+3] x B[cols tx*6..+5] over `len` reduction steps
// (A: reduction-major with row stride AS).
template <int AS = kAS>
__device__ __forceinline__ void tile_fma(const float* A, const float* B, int len, int ty, int tx,
                                         float (&acc)[4][6]) {
#pragma unroll 8
  for (int q = 0; q < len; ++q) {
    const float4 a = *reinterpret_cast<const float4*>(A + q * AS + ty * 4);
    const float2 b0 = *reinterpret_cast<const float2*>(B + q * kNT + tx * 6);
    const float2 b1 = *reinterpret_cast<const float2*>(B + q * kNT + tx * 6 + 2);
    const float2 b2 = *reinterpret_cast<const float2*>(B + q * kNT + tx * 6 + 4);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[6] = {b0.x, b0.y, b1.x, b1.y, b2.x, b2.y};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[i][c] = fmaf(av[i], bv[c], acc[i][c]);
  }
}

// smooth_eval for spectrum s of a tile, by a quad of lanes (the four lanes
// 4 (lane / 4) .. + 3 of a warp, mask qmask): lane l4 = lane % 4 of the quad
// takes the modes k = l4, l4 + 4, ...; the coefficients come from the tile's
// mode-major shared array (row stride AS), the twiddles from global memory.
// The butterfly leaves the same bits in all four lanes (each lane adds the
// same two partial sums, in either order), so a quad takes its Newton
// branches together.
template <int AS = kAS>
__device__ __forceinline__ void quad_smooth_eval(const float2* tw, const float* Cs, int s, int n,
                                                 int k_c, int J, float d, int l4, unsigned qmask,
                                                 float* s0, float* s1, float* s2) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  const float two_over_n = 2.0f / (float)n;
  int m = (l4 * J) % n;                             // (k J) mod n, k = l4 + 4 i
  const int step = (4 * J) % n;
  for (int k = l4; k <= k_c; k += 4, m = (m + step >= n) ? m + step - n : m + step) {
    float sp, cp;
    sincospif(two_over_n * (float)k * d, &sp, &cp);
    const float2 t = __ldg(&tw[m]);
    const float c = t.x * cp - t.y * sp;             // cos(2 pi k (J + d) / n)
    const float sn = t.y * cp + t.x * sp;            // sin(2 pi k (J + d) / n)
    const float qa = Cs[(2 * k) * AS + s], qb = Cs[(2 * k + 1) * AS + s];
    const float g = k == 0 ? 1.0f : 2.0f;
    const float w = 3.14159265358979f * two_over_n * (float)k;
    const float e = qa * c + qb * sn;
    a0 = fmaf(g, e, a0);
    a1 = fmaf(g * w, qb * c - qa * sn, a1);
    a2 = fmaf(-g * w * w, e, a2);
  }
  for (int o = 1; o <= 2; o <<= 1) {
    a0 += __shfl_xor_sync(qmask, a0, o);
    a1 += __shfl_xor_sync(qmask, a1, o);
    a2 += __shfl_xor_sync(qmask, a2, o);
  }
  *s0 = a0;
  *s1 = a1;
  *s2 = a2;
}

// 16-byte global-to-shared copies that bypass registers (cp.async, .cg: L2 only).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One kJC x kNT chunk of a row-major matrix (row stride `ld` floats) into a
// shared buffer, 16 bytes per copy: 768 copies, three per thread.
__device__ __forceinline__ void load_chunk_async(float* dst, const float* src, size_t ld,
                                                 int tid) {
#pragma unroll
  for (int u = 0; u < kJC * kNT / 4 / 256; ++u) {
    const int e = tid + u * 256, r = e / (kNT / 4), c4 = e % (kNT / 4);
    cp_async16(dst + 4 * e, src + (size_t)r * ld + 4 * c4);
  }
  cp_async_commit();
}

// The per-spectrum end of stage 2 for n_sp spectra (the first at global index
// s0): status, Newton refinement from the coefficients (Cs mode-major, row
// stride AS) and Eq. 35, from each spectrum's first window maximum (red_v,
// red_j: value and absolute bin). One quad of lanes per spectrum, so a warp
// runs eight spectra's Newton steps side by side; thread tid of the calling
// group of n_threads (a multiple of 32) is lane tid % 4 of quad tid / 4.
template <int AS>
__device__ __forceinline__ void tile_finish(const float* Cs, const float* red_v, const int* red_j,
                                            int n_sp, int s0, int n_spec, int n, int k_c, int j_lo,
                                            int j_hi, PeakGeom geom, const float2* tw,
                                            pdv_peak* out, int tid, int n_threads) {
  const int n_w = j_hi - j_lo + 1;
  const int lane = tid & 31, l4 = lane & 3;
  const unsigned qmask = 0xFu << (lane & ~3);
  for (int s = tid >> 2; s < n_sp; s += n_threads >> 2) {
    const int gs = s0 + s;
    if (gs >= n_spec) break;
    const float bv = red_v[s];
    const int J = red_j[s];
    pdv_peak r;
    r.x_peak = r.i_peak = r.curvature = r.beta = r.tau0 = NAN;
    r.j_max = (n_w >= 1) ? J : -1;
    r.status = PDV_PEAK_NO_PEAK;
    if (n_w >= 1 && bv > 0.0f) {
      if (J == j_lo || J == j_hi) {
        r.status = PDV_PEAK_EDGE;
      } else {
        float d = 0.f, q0, q1, q2;
        quad_smooth_eval<AS>(tw, Cs, s, n, k_c, J, d, l4, qmask, &q0, &q1, &q2);
        for (int it = 0; it < kPeakNewton && q2 < 0.0f; ++it) {
          const float nd = fminf(fmaxf(d - q1 / q2, -1.0f), 1.0f);
          const bool done = fabsf(nd - d) <= 1e-6f;
          d = nd;
          if (done) break;
          quad_smooth_eval<AS>(tw, Cs, s, n, k_c, J, d, l4, qmask, &q0, &q1, &q2);
        }
        peak_finish(r, J, d, q0, q2, 1.0f / (float)n, geom);
      }
    }
    if (l4 == 0) out[gs] = r;
  }
}

// Stage 2 of a tile of kTS spectra (the first at global index s0): smoothed
// window values (coefficients x G, Cs mode-major with row stride AS), the
// running first maximum per spectrum, then per spectrum the status, the Newton
// refinement and Eq. 35. Run by 256 threads (tid: 0..255; two groups of 256
// may run it side by side with their own buffers, as its block barriers
// match). Bs: two kJC x kNT buffers; red_v / red_j: kTS each.
template <int AS>
__device__ __forceinline__ void tile_peaks(const float* Cs, int s0, int n_spec, int n, int k_c,
                                           int j_lo, int j_hi, PeakGeom geom, const float2* tw,
                                           const float* G, int k2p, int nw_p, float* Bs,
                                           float* red_v, int* red_j, pdv_peak* out, int tid) {
  const int ty = tid >> 4, tx = tid & 15;
  const int n_w = j_hi - j_lo + 1;
  // ---- smoothed window values (tile x G), running first maximum per spectrum
  float best[4];
  int bj[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    best[i] = -INFINITY;
    bj[i] = 0x7fffffff;
  }
  // chunks run column tile by column tile, the next chunk of G copied into
  // the other shared buffer (cp.async) while this one is multiplied
  {
    const int nr = k2p / kJC, nchunks = nr * (nw_p / kNT);
    auto g_src = [&](int ch) {
      return G + (size_t)((ch % nr) * kJC) * nw_p + (ch / nr) * kNT;
    };
    float acc[4][6];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[i][c] = 0.0f;
    __syncthreads();                               // B buffers free
    if (nchunks) load_chunk_async(Bs, g_src(0), (size_t)nw_p, tid);
    for (int ch = 0; ch < nchunks; ++ch) {
      cp_async_wait_all();
      __syncthreads();                             // this chunk visible; the other buffer free
      if (ch + 1 < nchunks)
        load_chunk_async(Bs + ((ch + 1) & 1) * (kJC * kNT), g_src(ch + 1), (size_t)nw_p, tid);
      tile_fma<AS>(Cs + (ch % nr) * kJC * AS, Bs + (ch & 1) * (kJC * kNT), kJC, ty, tx, acc);
      if (ch % nr == nr - 1) {
        const int wp = (ch / nr) * kNT;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const int j = wp + tx * 6 + c;
          if (j < n_w) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (acc[i][c] > best[i]) {
                best[i] = acc[i][c];
                bj[i] = j_lo + j;
              }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 6; ++c) acc[i][c] = 0.0f;
      }
    }
  }
  // reduce over the 16 threads sharing ty (lanes 0-15 and 16-31 of a warp)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    for (int o = 8; o; o >>= 1) {
      const float ov = __shfl_xor_sync(kFull, best[i], o);
      const int oj = __shfl_xor_sync(kFull, bj[i], o);
      if (ov > best[i] || (ov == best[i] && oj < bj[i])) {
        best[i] = ov;
        bj[i] = oj;
      }
    }
    if (tx == 0) {
      red_v[ty * 4 + i] = best[i];
      red_j[ty * 4 + i] = bj[i];
    }
  }
  __syncthreads();
  tile_finish<AS>(Cs, red_v, red_j, kTS, s0, n_spec, n, k_c, j_lo, j_hi, geom, tw, out, tid, 256);
  __syncthreads();
}

__global__ void __launch_bounds__(256, 3) k_extract_tiled(
    const double* spec, int n_spec, int n, int k_c, int j_lo, int j_hi, PeakGeom geom,
    const float2* tw, const float* F, const float* G, int n_p, int k2p, int nw_p, pdv_peak* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TileSmem L = tile_layout(k2p);
  float* As = reinterpret_cast<float*>(smem + L.o_a);    // [kJC][kAS] spectra chunk (j-major)
  float* Bs = reinterpret_cast<float*>(smem + L.o_b);    // [kJC][kNT] F or G chunk
  float* Cs = reinterpret_cast<float*>(smem + L.o_c);    // [k2p][kAS] coefficients (mode-major)
  float* red_v = reinterpret_cast<float*>(smem + L.o_red);
  int* red_j = reinterpret_cast<int*>(red_v + kTS);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_tiles = (n_spec + kTS - 1) / kTS;

  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int s0 = tile * kTS;
    // ---- coefficients: Cs = tile x F, column passes of kNT
    for (int cp = 0; cp < k2p; cp += kNT) {
      float acc[4][6];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[i][c] = 0.0f;
      // the next chunk is in flight while this one is multiplied: F by
      // cp.async into the other shared buffer, the spectra as raw FP64 words in
      // registers (lane = bin of the chunk, warp + 8 u = spectrum), converted
      // to FP32 only after the products, so their loads overlap them
      double ra[kTS / 8];
      float pa[kTS / 8];
      auto fetch_a = [&](int j0) {
        const int gj = j0 + lane;
#pragma unroll
        for (int u = 0; u < kTS / 8; ++u) {
          const int gs = s0 + warp + 8 * u;
          ra[u] = (gs < n_spec && gj < n) ? spec[(size_t)gs * n + gj] : 0.0;
        }
      };
      auto convert_a = [&]() {
#pragma unroll
        for (int u = 0; u < kTS / 8; ++u) pa[u] = f64_to_f32(ra[u]);
      };
      fetch_a(0);
      convert_a();
      __syncthreads();                               // B buffers free (previous users done)
      load_chunk_async(Bs, F + cp, (size_t)k2p, tid);
      for (int j0 = 0, c = 0; j0 < n_p; j0 += kJC, ++c) {
        float* Bc = Bs + (c & 1) * (kJC * kNT);
        __syncthreads();                             // previous chunk's products done
#pragma unroll
        for (int u = 0; u < kTS / 8; ++u) As[lane * kAS + warp + 8 * u] = pa[u];
        cp_async_wait_all();
        __syncthreads();                             // As and this chunk of F visible
        if (j0 + kJC < n_p) {
          load_chunk_async(Bs + ((c + 1) & 1) * (kJC * kNT), F + (size_t)(j0 + kJC) * k2p + cp,
                           (size_t)k2p, tid);
          fetch_a(j0 + kJC);
        }
        tile_fma(As, Bc, kJC, ty, tx, acc);
        if (j0 + kJC < n_p) convert_a();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 6; ++c) Cs[(cp + tx * 6 + c) * kAS + ty * 4 + i] = acc[i][c];
    }
    tile_peaks<kAS>(Cs, s0, n_spec, n, k_c, j_lo, j_hi, geom, tw, G, k2p, nw_p, Bs, red_v, red_j,
                    out, tid);
  }
}

// ------------------------------------------------------------------ tensor-core extraction
// The first product (the DFT coefficients of a tile of kTcM = 128 spectra) on
// the tensor cores: tcgen05.mma kind::tf32 with both operands in shared memory
// (K-major, 128-byte swizzle) and FP32 accumulators in tensor memory (lane =
// spectrum, column = coefficient row).
//  * FP32 accuracy from TF32 operands: x = hi + lo with hi = x rounded to TF32
//    and lo = the remainder rounded to TF32, three products per step,
//    hi*hi + hi*lo + lo*hi; the dropped lo*lo and the rounding of lo are each
//    below 2^-22 of |x| |F|.
//  * The tensor core adds into its FP32 accumulator with truncation, so the
//    sums are kept short: hi*hi and the two correction products go to separate
//    accumulators, and every kTcG chunks (128 bins) both are added into the
//    coefficient array in FP32 (round to nearest) while the next group
//    accumulates into a second pair.
//  * The spectra are read as FP64, converted to FP32 in integer operations,
//    split and stored by the threads; the split cosine/sine matrix comes from a
//    table built once per call, by cp.async. Chunks of kTcKC bins alternate
//    between two shared buffers: while the tensor core multiplies one, the
//    threads fill the other, and mbarriers that the products' commits arrive
//    on free buffers and accumulator pairs. Every wait is bounded; a timeout
//    sets the error word, waits once more for the products in flight, frees
//    the tensor memory and returns.
//  * Stage 2: the smoothed window values W = C G (coefficients times the
//    window's cosine/sine matrix) are a second product on the tensor cores,
//    in passes of kTcN2 window bins with the coefficients split the same way
//    and their own pair of accumulators; each thread then scans its
//    spectrum's row of W in tensor memory for the first maximum, and one warp
//    per spectrum runs the Newton refinement and Eq. 35 on the CUDA cores.
constexpr int kTcM = 128;                  // spectra per tile: the products' M
constexpr int kTcKC = 32;                  // bins per chunk: one 128-byte row, four steps of K = 8
constexpr int kTcG = 4;                    // chunks an accumulator pair sums before it is added up
constexpr int kTcThreads = 512;
constexpr int kTcAS = kTcM + 4;            // row stride of the coefficient array
constexpr uint32_t kTcCols = 512;          // tensor-memory columns: two pairs of nt <= 128
constexpr int kTcN2 = 256;                 // most window bins in a pass of the second product
constexpr int kTcWaitLimit = 1 << 20;      // polls of an mbarrier before a wait gives up

struct TcSmem {
  size_t o_a, o_b, o_c, o_red, o_bar, bytes;
};

__host__ __device__ inline size_t align1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

// nt: the products' N (coefficient rows, a multiple of 16, <= 128); k2s: rows
// of the coefficient array and of G (a multiple of kJC, >= nt). Offsets from a
// 1024-byte aligned base (the launch adds 1 KB for that alignment).
__host__ __device__ inline TcSmem tc_layout(int nt, int k2s) {
  TcSmem L;
  const size_t a_tile = sizeof(float) * kTcM * kTcKC, b_tile = sizeof(float) * (size_t)nt * kTcKC;
  L.o_a = 0;                                         // [buffer][hi, lo] spectra tiles
  L.o_b = align1k(L.o_a + 4 * a_tile);               // [buffer][hi, lo] matrix tiles
  // the B tiles' space also holds stage 2's split coefficient tiles (2 a_tile)
  L.o_c = align1k(L.o_b + (4 * b_tile > 2 * a_tile ? 4 * b_tile : 2 * a_tile));
  L.o_red = L.o_c + sizeof(float) * (size_t)k2s * kTcAS;      // window maxima: 5 x kTcM pairs
  L.o_bar = (L.o_red + 5 * (sizeof(float) + sizeof(int)) * kTcM + 15) & ~(size_t)15;
  L.bytes = L.o_bar + 64;                            // five mbarriers, the tensor-memory address
  return L;
}

// byte offset of the 16 bytes holding bins 4 ch .. 4 ch + 3 of row r in a
// K-major tile with 128-byte rows: 8-row atoms of 1024 bytes, the 16-byte
// unit index XORed with the row within the atom (the 128-byte swizzle)
__device__ __forceinline__ uint32_t sw128(int r, int ch) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major with 128-byte swizzle: start
// address, leading offset 16 bytes (unused for this layout), stride 1024
// bytes between 8-row atoms, descriptor version 1 (bits 46-48), swizzle mode 2
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A B^T, M = kTcM, N from the instruction descriptor, K = 8
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the mbarrier tracks completion of every product this thread issued before
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kTcWaitLimit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
  return done != 0;
}

// 16 consecutive columns of this warp's 32 tensor-memory lanes, one lane per thread
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// FTh / FTl: [nt][n_k], row r = 2k the cosine and 2k + 1 the sine of
// 2 pi j k / n (zero for k > k_c or j >= n), split into TF32 hi + lo from FP64.
// GTh / GTl: [nw_p][k2s], the window matrix of k_peak_mats transposed (row =
// window bin, column = coefficient row), split the same way.
__global__ void k_peak_mats_tc(int n, int k_c, int n_k, int nt, int k2s, int j_lo, int n_w,
                               int nw_p, float* FTh, float* FTl, float* GTh, float* GTl) {
  const long long nF = (long long)nt * n_k, nG = (long long)k2s * nw_p;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nF + nG;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nF) {
      const int r = (int)(t / n_k), j = (int)(t % n_k), k = r >> 1;
      double v = 0.0;
      if (j < n && k <= k_c) {
        double sn, cs;
        sincospi(2.0 * (double)(((long long)j * k) % n) / n, &sn, &cs);
        v = (r & 1) ? sn : cs;
      }
      const float hi = __uint_as_float(to_tf32((float)v));
      FTh[t] = hi;
      FTl[t] = __uint_as_float(to_tf32((float)(v - (double)hi)));
    } else {
      const long long u = t - nF;
      const int j = (int)(u / k2s), r = (int)(u % k2s), k = r >> 1;
      double v = 0.0;
      if (j < n_w && k <= k_c && !(k == 0 && (r & 1))) {
        double sn, cs;
        sincospi(2.0 * (double)(((long long)(j_lo + j) * k) % n) / n, &sn, &cs);
        v = ((r & 1) ? sn : cs) * (k == 0 ? 1.0 : 2.0) / n;
      }
      const float hi = __uint_as_float(to_tf32((float)v));
      GTh[u] = hi;
      GTl[u] = __uint_as_float(to_tf32((float)(v - (double)hi)));
    }
  }
}

// Adds accumulator pair `set` (hi*hi and corrections, nt columns each) into
// Cs: warp w reads lanes 32 (w & 3) .. + 31 and every fourth group of 16 columns.
__device__ __forceinline__ void tc_flush(uint32_t tmem, int set, int nt, float* Cs, int warp,
                                         int lane) {
  const int q = warp & 3, row = q * 32 + lane;
  const uint32_t lanes = (uint32_t)(q * 32) << 16;
  for (int c0 = (warp >> 2) * 16; c0 < nt; c0 += 64) {
    uint32_t m[16], e[16];
    tc_ld16(tmem + lanes + (uint32_t)(set * 2 * nt + c0), m);
    tc_ld16(tmem + lanes + (uint32_t)(set * 2 * nt + nt + c0), e);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      Cs[(c0 + j) * kTcAS + row] += __uint_as_float(m[j]) + __uint_as_float(e[j]);
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_extract_tc(
    const double* spec, int n_spec, int n, int k_c, int j_lo, int j_hi, PeakGeom geom,
    const float2* tw, const float* FTh, const float* FTl, const float* GTh, const float* GTl,
    int n_k, int nt, int k2s, int nw_p, pdv_peak* out, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the swizzled tiles need 1024-byte alignment of their shared-memory addresses
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const TcSmem L = tc_layout(nt, k2s);
  unsigned char* As = smem + L.o_a;
  unsigned char* Bsm = smem + L.o_b;
  float* Cs = reinterpret_cast<float*>(smem + L.o_c);
  float* red_v = reinterpret_cast<float*>(smem + L.o_red);         // [kTcM] first window maximum
  int* red_j = reinterpret_cast<int*>(red_v + kTcM);
  float* red4_v = reinterpret_cast<float*>(red_j + kTcM);          // [4][kTcM] per column group
  int* red4_j = reinterpret_cast<int*>(red4_v + 4 * kTcM);
  // [0, 1]: buffers; [2, 3]: accumulator pairs; [4]: the second product
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.o_bar);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + L.o_bar + 48);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t a_tile = sizeof(float) * kTcM * kTcKC, b_tile = sizeof(float) * (size_t)nt * kTcKC;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(taddr_s)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_s;
  // F32 accumulator, TF32 A and B, both K-major, N = nt, M = kTcM
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) |
                         ((uint32_t)(kTcM >> 4) << 24);
  uint32_t ph[5] = {0u, 0u, 0u, 0u, 0u};            // parity of each mbarrier's next completion
  const int n_w = j_hi - j_lo + 1;
  int fail = 0;
  const int n_chunks = n_k / kTcKC, n_groups = (n_chunks + kTcG - 1) / kTcG;
  const int n_tiles = (n_spec + kTcM - 1) / kTcM;
  const int r = tid >> 2, qb = tid & 3;             // A fill: row r, 16-byte units qb and qb + 4
  auto wait = [&](int i) {
    const bool ok = mbar_wait(&bar[i], ph[i]);
    ph[i] ^= 1u;
    return ok;
  };
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int s0 = tile * kTcM, gs = s0 + r;
    const double* row = spec + (size_t)(gs < n_spec ? gs : 0) * n;
    for (int e = tid; e < k2s * kTcM; e += kTcThreads) Cs[(e / kTcM) * kTcAS + e % kTcM] = 0.0f;
    // a thread's 8 bins of a chunk are bins 4 qb .. 4 qb + 3 and 16 + 4 qb .. 16 + 4 qb + 3
    // of its row, so the four threads of a row read 128 contiguous bytes per load. With
    // every row on a 16-byte boundary (n even, aligned base) the loads are 16 bytes wide:
    // a warp's load then asks for whole 32-byte sectors, each once
    double ra[8];
    const bool v2 = ((n & 1) == 0) && ((reinterpret_cast<uintptr_t>(spec) & 15) == 0);
    auto fetch = [&](int c) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j0 = c * kTcKC + 16 * u + 4 * qb;
        if (v2) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = j0 + 2 * h;
            double2 x = make_double2(0.0, 0.0);
            if (gs < n_spec && j < n) x = __ldcs(reinterpret_cast<const double2*>(row + j));
            ra[4 * u + 2 * h] = x.x;
            ra[4 * u + 2 * h + 1] = x.y;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            ra[4 * u + i] = (gs < n_spec && j0 + i < n) ? __ldcs(row + j0 + i) : 0.0;
        }
      }
    };
    fetch(0);
    for (int c = 0; c < n_chunks; ++c) {
      const int b = c & 1, g = c / kTcG, set = g & 1;
      const bool first = c % kTcG == 0;
      // Each thread waits on the mbarriers for itself and writes only its own pieces of the
      // buffers; a wait that gave up reaches every thread at the block barrier before the
      // products, the one barrier a chunk needs
      int lfail = 0;
      if (c >= 2 && !wait(b)) lfail = 1;             // buffer b's products (chunk c - 2) done
      if (first && g >= 2) {                         // pair `set` summed group g - 2: add it up
        // the flush's tensor-memory loads are warp-wide (.sync.aligned): a warp flushes
        // only if every lane saw the pair complete
        if (!__all_sync(kFull, wait(2 + set))) {
          lfail = 1;
        } else {
          tc_fence_after();
          tc_flush(tmem, set, nt, Cs, warp, lane);
          tc_fence_before();
        }
      }
      unsigned char* Ah = As + (2 * b) * a_tile;
      unsigned char* Al = Ah + a_tile;
      unsigned char* Bh = Bsm + (2 * b) * b_tile;
      unsigned char* Bl = Bh + b_tile;
      // the matrix chunk: rows 0..nt-1, bins c kTcKC .. + kTcKC, 16 bytes (4 bins) a copy
      for (int e = tid; e < nt * (kTcKC / 4); e += kTcThreads) {
        const int rr = e >> 3, k4 = e & 7;
        const size_t src = (size_t)rr * n_k + (size_t)c * kTcKC + 4 * k4;
        cp_async16(Bh + sw128(rr, k4), FTh + src);
        cp_async16(Bl + sw128(rr, k4), FTl + src);
      }
      cp_async_commit();
      // the spectra chunk: convert, split, 4 bins of one row a 16-byte store
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float x = f64_to_f32(ra[4 * u + t]);
          hi[t] = to_tf32(x);
          lo[t] = to_tf32(x - __uint_as_float(hi[t]));
        }
        const uint32_t off = sw128(r, qb + 4 * u);
        *reinterpret_cast<uint4*>(Ah + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(Al + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      if (c + 1 < n_chunks) fetch(c + 1);           // in flight during this chunk's products
      cp_async_wait_all();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      const int any_fail = __syncthreads_or(lfail);
      tc_fence_after();
      if (any_fail) {
        fail = 1;
        break;
      }
      if (tid == 0) {
        const uint32_t ah = smem_addr(Ah), al = smem_addr(Al), bh = smem_addr(Bh), bl = smem_addr(Bl);
        const uint32_t dm = tmem + (uint32_t)(set * 2 * nt), dc = dm + (uint32_t)nt;
#pragma unroll
        for (int ks = 0; ks < kTcKC / 8; ++ks) {
          const uint32_t o = (uint32_t)ks * 32;     // 8 bins along the 128-byte row
          const uint32_t acc = (first && ks == 0) ? 0u : 1u;
          tc_mma(dm, tc_desc(ah + o), tc_desc(bh + o), idesc, acc);
          tc_mma(dc, tc_desc(ah + o), tc_desc(bl + o), idesc, acc);
          tc_mma(dc, tc_desc(al + o), tc_desc(bh + o), idesc, 1u);
        }
        tc_commit(&bar[b]);
        if (c % kTcG == kTcG - 1 || c == n_chunks - 1) tc_commit(&bar[2 + set]);
      }
    }
    if (fail) break;
    // the buffers' outstanding completions, then the pairs not yet added up
    bool ok = wait(0);
    if (n_chunks > 1) ok = wait(1) && ok;
    for (int g = n_groups >= 2 ? n_groups - 2 : 0; g < n_groups; ++g) {
      ok = wait(2 + (g & 1)) && ok;
      if (__syncthreads_or(!ok)) {
        fail = 1;
        break;
      }
      tc_fence_after();
      tc_flush(tmem, g & 1, nt, Cs, warp, lane);
    }
    if (fail) break;
    tc_fence_before();
    __syncthreads();
    // ---- stage 2: W = C G in passes of kTcN2 window bins, K-chunks of kTcKC
    // coefficient rows; the split tiles reuse the spectra tiles' buffer
    const int q = warp & 3, cg = warp >> 2, srow = q * 32 + lane;   // scan: row srow, columns cg + 4 i
    float bv = -INFINITY;
    int bjx = 0x7fffffff;
    unsigned char* A2h = Bsm;                        // split coefficients: 128 rows x 32 coefficient rows
    unsigned char* A2l = Bsm + a_tile;
    unsigned char* B2h = As;                         // split window matrix: up to kTcN2 rows
    unsigned char* B2l = As + sizeof(float) * kTcN2 * kTcKC;     // 32 KB further: 256 rows x 128 B
    for (int j0 = 0; j0 < nw_p && !fail; j0 += kTcN2) {
      const int n2 = nw_p - j0 < kTcN2 ? nw_p - j0 : kTcN2;     // this pass's N (a multiple of 16)
      const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n2 >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);
      for (int kc = 0; kc < k2s; kc += kTcKC) {
        for (int e = tid; e < n2 * (kTcKC / 4); e += kTcThreads) {
          const int rr = e >> 3, k4 = e & 7;
          const size_t src = (size_t)(j0 + rr) * k2s + kc + 4 * k4;
          cp_async16(B2h + sw128(rr, k4), GTh + src);
          cp_async16(B2l + sw128(rr, k4), GTl + src);
        }
        cp_async_commit();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float x = Cs[(kc + 8 * qb + 4 * u + t) * kTcAS + r];
            hi[t] = to_tf32(x);
            lo[t] = to_tf32(x - __uint_as_float(hi[t]));
          }
          const uint32_t off = sw128(r, 2 * qb + u);
          *reinterpret_cast<uint4*>(A2h + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(A2l + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
          const uint32_t ah = smem_addr(A2h), al = smem_addr(A2l), bh = smem_addr(B2h),
                         bl = smem_addr(B2l);
#pragma unroll
          for (int ks = 0; ks < kTcKC / 8; ++ks) {
            const uint32_t o = (uint32_t)ks * 32;
            const uint32_t acc = (kc == 0 && ks == 0) ? 0u : 1u;
            tc_mma(tmem, tc_desc(ah + o), tc_desc(bh + o), idesc2, acc);
            tc_mma(tmem + kTcN2, tc_desc(ah + o), tc_desc(bl + o), idesc2, acc);
            tc_mma(tmem + kTcN2, tc_desc(al + o), tc_desc(bh + o), idesc2, 1u);
          }
          tc_commit(&bar[4]);
        }
        if (__syncthreads_or(!wait(4))) {            // the split tiles are free again
          fail = 1;
          break;
        }
      }
      if (fail) break;
      tc_fence_after();
      // this thread's groups of 16 window bins of spectrum srow (groups cg, cg + 4, ...):
      // the first maximum, in bin order
      for (int c0 = cg * 16; c0 < n2; c0 += 64) {
        uint32_t m[16], e[16];
        const uint32_t a = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        tc_ld16(a, m);
        tc_ld16(a + kTcN2, e);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jj = j0 + c0 + j;
          const float v = __uint_as_float(m[j]) + __uint_as_float(e[j]);
          if (jj < n_w && v > bv) {
            bv = v;
            bjx = j_lo + jj;
          }
        }
      }
      tc_fence_before();
      __syncthreads();                               // before the next pass writes the accumulators
    }
    if (fail) break;
    red4_v[cg * kTcM + srow] = bv;
    red4_j[cg * kTcM + srow] = bjx;
    __syncthreads();
    if (tid < kTcM) {                                // first maximum over the four column groups
      float v = red4_v[tid];
      int jx = red4_j[tid];
      for (int g = 1; g < 4; ++g) {
        const float ov = red4_v[g * kTcM + tid];
        const int oj = red4_j[g * kTcM + tid];
        if (ov > v || (ov == v && oj < jx)) {
          v = ov;
          jx = oj;
        }
      }
      red_v[tid] = v;
      red_j[tid] = jx;
    }
    __syncthreads();
    tile_finish<kTcAS>(Cs, red_v, red_j, kTcM, s0, n_spec, n, k_c, j_lo, j_hi, geom, tw, out, tid,
                       kTcThreads);
    __syncthreads();                                 // Cs and the tiles free for the next tile
  }
  if (fail) {
    if (tid == 0) atomicExch(err, 1);
    // the products still in flight, once more with a bound, before the tensor memory is freed
    for (int i = 0; i < 5; ++i) (void)mbar_wait(&bar[i], ph[i]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols)
                 : "memory");
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
  const long long total = (long long)n_sets * ((n_bins + kRun - 1) / kRun);
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
                           PeakGeom geom, const float2* d_tw, pdv_peak* d_out, int grid,
                           cudaStream_t st) {
  k_extract<<<grid, kPeakThreads, peak_smem(n, k_c), st>>>(d_spec, n_spec, n, k_c, j_lo, j_hi,
                                                            geom, d_tw, d_out);
  return cudaGetLastError();
}

}  // namespace pdv

namespace pdv {

bool peak_tiled(int k_c) { return pad_to(2 * (k_c + 1), kNT) <= kTileMaxK2; }

size_t peak_mats_bytes(int n, int k_c, int n_w) {
  const size_t k2p = pad_to(2 * (k_c + 1), kNT), n_p = pad_to(n, kJC);
  const size_t nw_p = pad_to(n_w > 0 ? n_w : 0, kNT);
  return sizeof(float) * (n_p * k2p + k2p * nw_p) + 16;
}

cudaError_t tiled_occupancy(int k_c, int* blocks_per_sm) {
  const size_t sm = tile_layout(pad_to(2 * (k_c + 1), kNT)).bytes;
  cudaError_t e = cudaFuncSetAttribute(k_extract_tiled,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_extract_tiled, 256, sm);
}

cudaError_t launch_extract_tiled(const double* d_spec, int n_spec, int n, int k_c, int j_lo,
                                 int j_hi, PeakGeom geom, const float2* d_tw, float* d_mats,
                                 pdv_peak* d_out,
                                 int blocks_per_sm, int sm_count, cudaStream_t st,
                                 cudaEvent_t e0, cudaEvent_t e1) {
  const int k2p = pad_to(2 * (k_c + 1), kNT), n_p = pad_to(n, kJC);
  const int n_w = j_hi - j_lo + 1 > 0 ? j_hi - j_lo + 1 : 0;
  const int nw_p = pad_to(n_w, kNT);
  float* F = d_mats;
  float* G = d_mats + (size_t)n_p * k2p;
  const long long nm = (long long)n_p * k2p + (long long)k2p * nw_p;
  k_peak_mats<<<(int)std::min<long long>((nm + 255) / 256, 4096), 256, 0, st>>>(
      n, k_c, n_p, k2p, j_lo, n_w, nw_p, F, G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_tiles = (n_spec + kTS - 1) / kTS;
  const int grid = std::min(n_tiles, blocks_per_sm * sm_count);
  if (e0) cudaEventRecord(e0, st);
  k_extract_tiled<<<grid, 256, tile_layout(k2p).bytes, st>>>(
      d_spec, n_spec, n, k_c, j_lo, j_hi, geom, d_tw, F, G, n_p, k2p, nw_p, d_out);
  if (e1) cudaEventRecord(e1, st);
  return cudaGetLastError();
}

// ---- tensor-core extraction
static int tc_nt(int k_c) { return pad_to(2 * (k_c + 1), 16); }
static int tc_k2s(int k_c) { return pad_to(tc_nt(k_c), kJC); }

// the layout plus 1 KB for aligning its base, and at least half an SM's
// shared memory so that one block (which holds all 512 tensor-memory
// columns) runs per SM
size_t tc_smem(int k_c) {
  const size_t b = tc_layout(tc_nt(k_c), tc_k2s(k_c)).bytes + 1024;
  return b > 120 * 1024 ? b : 120 * 1024;
}

bool peak_tc(int k_c, int max_smem) {
  return tc_nt(k_c) <= 128 && tc_smem(k_c) <= (size_t)max_smem;
}

size_t peak_mats_tc_bytes(int n, int k_c, int n_w) {
  const size_t nt = tc_nt(k_c), k2s = tc_k2s(k_c), n_k = pad_to(n, kTcKC);
  const size_t nw_p = pad_to(n_w > 0 ? n_w : 0, 16);
  return sizeof(float) * (2 * nt * n_k + 2 * nw_p * k2s) + 64;
}

cudaError_t tc_occupancy(int k_c, int* blocks_per_sm) {
  const size_t sm = tc_smem(k_c);
  cudaError_t e = cudaFuncSetAttribute(k_extract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_extract_tc, kTcThreads, sm);
  if (*blocks_per_sm > 1) *blocks_per_sm = 1;       // a block holds every tensor-memory column
  return e;
}

cudaError_t launch_extract_tc(const double* d_spec, int n_spec, int n, int k_c, int j_lo, int j_hi,
                              PeakGeom geom, const float2* d_tw, float* d_mats, pdv_peak* d_out,
                              int* d_err, int blocks_per_sm, int sm_count, cudaStream_t st,
                              cudaEvent_t e0, cudaEvent_t e1) {
  const int nt = tc_nt(k_c), k2s = tc_k2s(k_c), n_k = pad_to(n, kTcKC);
  const int n_w = j_hi - j_lo + 1 > 0 ? j_hi - j_lo + 1 : 0;
  const int nw_p = pad_to(n_w, 16);
  float* FTh = d_mats;
  float* FTl = FTh + (size_t)nt * n_k;
  float* GTh = FTl + (size_t)nt * n_k;
  float* GTl = GTh + (size_t)nw_p * k2s;
  const long long nm = 2LL * nt * n_k + (long long)k2s * nw_p;
  k_peak_mats_tc<<<(int)std::min<long long>((nm + 255) / 256, 4096), 256, 0, st>>>(
      n, k_c, n_k, nt, k2s, j_lo, n_w, nw_p, FTh, FTl, GTh, GTl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_tiles = (n_spec + kTcM - 1) / kTcM;
  const int grid = std::min(n_tiles, blocks_per_sm * sm_count);
  if (e0) cudaEventRecord(e0, st);
  k_extract_tc<<<grid, kTcThreads, tc_smem(k_c), st>>>(d_spec, n_spec, n, k_c, j_lo, j_hi, geom,
                                                       d_tw, FTh, FTl, GTh, GTl, n_k, nt, k2s, nw_p,
                                                       d_out, d_err);
  if (e1) cudaEventRecord(e1, st);
  return cudaGetLastError();
}

}  // namespace pdv

