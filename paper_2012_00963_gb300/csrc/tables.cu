// tables.cu — FP64 table builds on the device.
//
//  * cumulative mass fraction of the velocity profile at uniform velocity
//    nodes (Eq. 20, z = v t; the optical depth above the surface is
//    T = tau_tot S, Eq. 10 and Eq. 24), with an integer guide table;
//  * integer inverse CDF of the phase function p(theta) sin(theta) (Eq. 13);
//  * size-averaged Mie phase function and efficiencies (Eq. 12-14, Eq. 21),
//    from the series of Bohren & Huffman (1983, ch. 4).
#include <math.h>

#include "pdv_internal.cuh"

namespace pdv {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

struct Cplx {
  double re, im;
};
__device__ __forceinline__ Cplx cx(double r, double i) { return Cplx{r, i}; }
__device__ __forceinline__ Cplx operator+(Cplx a, Cplx b) { return cx(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ Cplx operator-(Cplx a, Cplx b) { return cx(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ Cplx operator*(Cplx a, Cplx b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ Cplx operator*(double s, Cplx a) { return cx(s * a.re, s * a.im); }
// Smith's algorithm for complex division (avoids overflow of |b|^2).
__device__ __forceinline__ Cplx operator/(Cplx a, Cplx b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return cx((a.re + a.im * r) / den, (a.im - a.re * r) / den);
  }
  const double r = b.re / b.im, den = b.re * r + b.im;
  return cx((a.re * r + a.im) / den, (a.im * r - a.re) / den);
}
__device__ __forceinline__ double cnorm(Cplx a) { return a.re * a.re + a.im * a.im; }

// ------------------------------------------------------------------ mass table
struct Profile {
  int kind;
  double beta, v_fs, v_bot, v_top, E;
  const double* pv;
  const double* pf;
  const double* cum;
  int n;
};

// Cumulative mass fraction S(v) in [0, 1].
__device__ double profile_cdf(const Profile& P, double v) {
  if (v <= P.v_bot) return 0.0;
  if (v >= P.v_top) return 1.0;
  if (P.kind == PDV_PROFILE_EXPONENTIAL) return -expm1(-P.beta * (v / P.v_fs - 1.0)) / P.E;
  int lo = 0, hi = P.n - 2;                 // segment with pv[i] <= v
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.pv[mid] <= v) lo = mid; else hi = mid - 1;
  }
  const double h = P.pv[lo + 1] - P.pv[lo];
  const double k = (P.pf[lo + 1] - P.pf[lo]) / h;
  const double x = v - P.pv[lo];
  return (P.cum[lo] + P.pf[lo] * x + 0.5 * k * x * x) / P.cum[P.n - 1];
}

// Trapezoid cumulative mass of a tabulated dm/dv (exact for piecewise-linear).
__global__ void k_profile_cum(const double* pv, const double* pf, int n, double* cum) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double c = 0.0;
  cum[0] = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    c = dadd(c, dmul(dmul(0.5, dadd(pf[i], pf[i + 1])), pv[i + 1] - pv[i]));
    cum[i + 1] = c;
  }
}

__global__ void k_mass_nodes(Profile P, int n_v, unsigned long long* Sq, double* Sd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_v) return;
  const double dv = (P.v_top - P.v_bot) / n_v;
  double s;
  if (j == 0) s = 0.0;
  else if (j == n_v) s = 1.0;
  else s = profile_cdf(P, P.v_bot + j * dv);
  Sd[j] = s;
  unsigned long long q = (unsigned long long)llrint(s * kTwo62);
  if (j == 0) q = 0ull;
  if (j == n_v || q > kOneQ) q = (j == n_v) ? kOneQ : q;
  Sq[j] = q;
}

__global__ void k_mass_slopes(const unsigned long long* Sq, int n_v, double dv, float* w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_v) return;
  const unsigned long long dq = Sq[j + 1] - Sq[j];
  w[j] = dq ? (float)(dv / (double)dq) : 0.0f;
}

// G[k] = largest j in [0, n_v - 1] with Sq_j <= k 2^g_shift.
__global__ void k_mass_guide(const unsigned long long* Sq, int n_v, int n_g, int g_shift,
                             unsigned short* G) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n_g) return;
  const unsigned long long target = (k == n_g) ? kOneQ : ((unsigned long long)k << g_shift);
  int lo = 0, hi = n_v - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (Sq[mid] <= target) lo = mid; else hi = mid - 1;
  }
  G[k] = (unsigned short)lo;
}

cudaError_t build_mass_table(int kind, double beta, double v_fs, double v_bot, double v_top,
                             const double* d_prof_v, const double* d_prof_f, int prof_n,
                             double* d_prof_cum, int n_v, CloudTables* t, cudaStream_t st) {
  Profile P;
  P.kind = kind;
  P.beta = beta;
  P.v_fs = v_fs;
  P.v_bot = v_bot;
  P.v_top = v_top;
  P.E = (kind == PDV_PROFILE_EXPONENTIAL) ? -expm1(-beta * (v_top / v_fs - 1.0)) : 1.0;
  P.pv = d_prof_v;
  P.pf = d_prof_f;
  P.cum = d_prof_cum;
  P.n = prof_n;
  if (kind == PDV_PROFILE_TABULATED) k_profile_cum<<<1, 1, 0, st>>>(d_prof_v, d_prof_f, prof_n, d_prof_cum);
  k_mass_nodes<<<(n_v + 1 + 255) / 256, 256, 0, st>>>(P, n_v, t->Sq, t->Sd);
  k_mass_slopes<<<(n_v + 255) / 256, 256, 0, st>>>(t->Sq, n_v, (v_top - v_bot) / n_v, t->w);
  k_mass_guide<<<(t->n_g + 1 + 255) / 256, 256, 0, st>>>(t->Sq, n_v, t->n_g, t->g_shift, t->G);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ phase CDF
__global__ void k_phase_trap(const double* th, const double* p, int n, double* work) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const double a = dmul(p[i], sin(th[i]));
  const double b = dmul(p[i + 1], sin(th[i + 1]));
  work[i] = dmul(dmul(0.5, dadd(a, b)), th[i + 1] - th[i]);
}

// Prefix sum of the trapezoids by one block in a fixed order (chunk sums,
// then a sequential scan of the chunk totals): deterministic run to run.
// work[n-1 + i] receives the cumulative C_i.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_phase_prefix(double* work, int n) {
  __shared__ double tot[kScanThreads];
  const int m = n - 1;                                  // number of trapezoids
  const int chunk = (m + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * chunk, e = min(b + chunk, m);
  double s = 0.0;
  for (int i = b; i < e; ++i) s = dadd(s, work[i]);
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int t = 0; t < kScanThreads; ++t) {
      const double v = tot[t];
      tot[t] = run;                                     // exclusive prefix of chunks
      run = dadd(run, v);
    }
  }
  __syncthreads();
  double* cum = work + m;
  double c = tot[threadIdx.x];
  if (threadIdx.x == 0) cum[0] = 0.0;
  for (int i = b; i < e; ++i) {
    c = dadd(c, work[i]);
    cum[i + 1] = c;
  }
}

__global__ void k_phase_quant(const double* work, const double* th, int n, unsigned* Cq,
                              float* thpi, double* thd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* cum = work + (n - 1);
  const double total = cum[n - 1];
  unsigned q = (unsigned)floor(cum[i] / total * 16777216.0 + 0.5);
  if (i == 0) q = 0u;
  if (i == n - 1) q = 16777216u;
  Cq[i] = q;
  thpi[i] = (float)(th[i] / 3.14159265358979323846);
  thd[i] = th[i];
}

// Slopes of the inverse CDF inside each bin: dthpi in half turns per CDF unit
// (the coarse-table walk), and the FP32 walk's node record (Cq_i, slope in
// radians per CDF unit), both from FP64.
__global__ void k_phase_slopes(const unsigned* Cq, const double* th, int n, float* dthpi,
                               uint2* node) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned dc = i == n - 1 ? 0u : Cq[i + 1] - Cq[i];
  const double dth = i == n - 1 ? 0.0 : th[i + 1] - th[i];
  dthpi[i] = dc ? (float)(dth / 3.14159265358979323846 / (double)dc) : 0.0f;
  node[i] = make_uint2(Cq[i], __float_as_uint(dc ? (float)(dth / (double)dc) : 0.0f));
}

// Gp[c] = largest i in [0, n-2] with Cq_i <= c 2^(24 - kGuidePhaseLog).
__global__ void k_phase_guide(const unsigned* Cq, int n, unsigned short* Gp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_gp = 1 << kGuidePhaseLog;
  if (c > n_gp) return;
  const unsigned target = (unsigned)c << (24 - kGuidePhaseLog);
  int lo = 0, hi = n - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (Cq[mid] <= target) lo = mid; else hi = mid - 1;
  }
  Gp[c] = (unsigned short)lo;
}

// Mean cosine of the sampled law (uniform theta inside each CDF bin): terms
// in parallel, one block, fixed-order tree reduction.
__global__ void __launch_bounds__(kScanThreads) k_phase_gtab(const unsigned* Cq, const double* th,
                                                             int n, double* g) {
  __shared__ double part[kScanThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i + 1 < n; i += kScanThreads) {
    const double dc = (double)(Cq[i + 1] - Cq[i]) / 16777216.0;
    s += dc * (sin(th[i + 1]) - sin(th[i])) / (th[i + 1] - th[i]);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = kScanThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *g = part[0];
}

cudaError_t build_phase_cdf(const double* d_theta, const double* d_p, int n, double* d_work,
                            CloudTables* t, double* d_gtab, cudaStream_t st) {
  const int nb = (n + 255) / 256;
  k_phase_trap<<<nb, 256, 0, st>>>(d_theta, d_p, n, d_work);
  k_phase_prefix<<<1, kScanThreads, 0, st>>>(d_work, n);
  k_phase_quant<<<nb, 256, 0, st>>>(d_work, d_theta, n, t->Cq, t->thpi, t->th_d);
  k_phase_slopes<<<nb, 256, 0, st>>>(t->Cq, d_theta, n, t->dthpi, t->node);
  k_phase_guide<<<((1 << kGuidePhaseLog) + 1 + 255) / 256, 256, 0, st>>>(t->Cq, n, t->Gp);
  k_phase_gtab<<<1, kScanThreads, 0, st>>>(t->Cq, d_theta, n, d_gtab);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Mie
// Size nodes: Gauss–Legendre in y = ln d over ln d_m +- 6 sigma, weighted by
// the number log-normal density of Eq. 21 (one node when sigma = 0).
__global__ void k_mie_nodes(int n, double d_m, double sigma, double wavelength, double* x,
                            double* wt, double* dd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double pi = 3.14159265358979323846;
  if (n == 1) {
    x[0] = pi * d_m / wavelength;
    wt[0] = 1.0;
    dd[0] = d_m;
    return;
  }
  double r = cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = r;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (r * p1 - p0) / (r * r - 1.0);
    const double dr = p1 / dp;
    r -= dr;
    if (fabs(dr) < 1e-16) break;
  }
  const double wgl = 2.0 / ((1.0 - r * r) * dp * dp);
  const double half = 6.0 * sigma;
  const double y = log(d_m) + half * r;
  const double t = (y - log(d_m)) / sigma;
  wt[i] = half * wgl * exp(-0.5 * t * t) / (sqrt(2.0 * pi) * sigma);
  dd[i] = exp(y);
  x[i] = pi * dd[i] / wavelength;
}

__host__ __device__ inline int mie_nmax(double x) {
  int n = (int)floor(x + 4.0 * cbrt(x) + 2.0);
  return n < 1 ? 1 : n;
}

// One thread per size: a_n, b_n with D_n(mx) by downward recurrence (kept only
// for n <= nmax) and Riccati–Bessel psi_n, chi_n by upward recurrence.
// q4[i] = (Q_ext, Q_sca, g Q_sca, nmax).
__global__ void k_mie_coeffs(int n_size, double mre, double mim, const double* xs,
                             long long ab_stride, Cplx* ab, long long d_stride, Cplx* dwork,
                             double* q4) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_size) return;
  const double x = xs[i];
  const Cplx m = cx(mre, mim);
  const Cplx mx = x * m;
  const int nmax = mie_nmax(x);
  int nstart = (int)ceil(sqrt(cnorm(mx)));
  if (nstart < nmax) nstart = nmax;
  nstart += 16;
  Cplx* D = dwork + (size_t)i * d_stride;   // D[n] = D_n(mx), n = 0..nmax
  Cplx* A = ab + (size_t)i * ab_stride;     // a_n at A[2n], b_n at A[2n+1], n = 1..nmax
  Cplx d = cx(0.0, 0.0);                    // D_nstart = 0
  for (int n = nstart; n >= 1; --n) {
    const Cplx nmx = cx(n, 0.0) / mx;
    d = nmx - cx(1.0, 0.0) / (d + nmx);     // D_{n-1}
    if (n - 1 <= nmax) D[n - 1] = d;
  }
  double psi_prev = cos(x), psi = sin(x), chi_prev = -sin(x), chi = cos(x);
  Cplx xi = cx(psi, -chi);
  double sext = 0.0, ssca = 0.0, gsum = 0.0;
  Cplx a_prev = cx(0, 0), b_prev = cx(0, 0);
  for (int n = 1; n <= nmax; ++n) {
    const double psi_n = (2.0 * n - 1.0) / x * psi - psi_prev;
    const double chi_n = (2.0 * n - 1.0) / x * chi - chi_prev;
    const Cplx xi_n = cx(psi_n, -chi_n);
    const Cplx da = D[n] / m + cx(n / x, 0.0);
    const Cplx db = m * D[n] + cx(n / x, 0.0);
    const Cplx an = (psi_n * da - cx(psi, 0.0)) / (da * xi_n - xi);
    const Cplx bn = (psi_n * db - cx(psi, 0.0)) / (db * xi_n - xi);
    A[2 * n] = an;
    A[2 * n + 1] = bn;
    const double fn = 2.0 * n + 1.0;
    sext += fn * (an.re + bn.re);
    ssca += fn * (cnorm(an) + cnorm(bn));
    if (n > 1) {
      const double k = n - 1.0;
      // Re(a_{n-1} a_n* + b_{n-1} b_n*) and Re(a_{n-1} b_{n-1}*)
      gsum += k * (k + 2.0) / (k + 1.0) *
                  (a_prev.re * an.re + a_prev.im * an.im + b_prev.re * bn.re + b_prev.im * bn.im) +
              (2.0 * k + 1.0) / (k * (k + 1.0)) * (a_prev.re * b_prev.re + a_prev.im * b_prev.im);
    }
    a_prev = an;
    b_prev = bn;
    psi_prev = psi; psi = psi_n;
    chi_prev = chi; chi = chi_n;
    xi = xi_n;
  }
  {
    const double k = nmax;
    gsum += (2.0 * k + 1.0) / (k * (k + 1.0)) * (a_prev.re * b_prev.re + a_prev.im * b_prev.im);
  }
  const double qext = 2.0 / (x * x) * sext;
  const double qsca = 2.0 / (x * x) * ssca;
  q4[4 * i + 0] = qext;
  q4[4 * i + 1] = qsca;
  q4[4 * i + 2] = 4.0 / (x * x) * gsum;     // g Q_sca
  q4[4 * i + 3] = (double)nmax;
}

// |S1|^2 + |S2|^2 at every angle for every size, times the size weight and
// lambda^2 / (8 pi^2) (so that p integrates to <C_sca>).
__global__ void k_mie_angles(int n_size, int n_angle, const double* xs, const double* wt,
                             long long ab_stride, const Cplx* ab, double wavelength,
                             double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= n_angle || i >= n_size) return;
  const double pi = 3.14159265358979323846;
  const double th = pi * (double)j / (double)(n_angle - 1);
  const double mu = cos(th);
  const Cplx* A = ab + (size_t)i * ab_stride;
  const int nmax = mie_nmax(xs[i]);
  double pi_prev = 0.0, pi_n = 1.0;
  Cplx S1 = cx(0, 0), S2 = cx(0, 0);
  for (int n = 1; n <= nmax; ++n) {
    const double tau_n = n * mu * pi_n - (n + 1.0) * pi_prev;
    const double fn = (2.0 * n + 1.0) / ((double)n * (n + 1.0));
    const Cplx an = A[2 * n], bn = A[2 * n + 1];
    S1 = S1 + fn * (pi_n * an + tau_n * bn);
    S2 = S2 + fn * (tau_n * an + pi_n * bn);
    const double pi_next = ((2.0 * n + 1.0) / n) * mu * pi_n - ((n + 1.0) / n) * pi_prev;
    pi_prev = pi_n;
    pi_n = pi_next;
  }
  out[(size_t)i * n_angle + j] =
      wt[i] * wavelength * wavelength / (8.0 * pi * pi) * (cnorm(S1) + cnorm(S2));
}

// Sum over sizes in fixed order (deterministic), theta grid.
__global__ void k_mie_reduce(int n_size, int n_angle, const double* out, double* theta, double* p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_angle) return;
  double s = 0.0;
  for (int i = 0; i < n_size; ++i) s += out[(size_t)i * n_angle + j];
  p[j] = s;
  theta[j] = 3.14159265358979323846 * (double)j / (double)(n_angle - 1);
}

__global__ void k_mie_scalars(int n_size, const double* wt, const double* dd, const double* q4,
                              double* q3) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double A2 = 0, Aext = 0, Asca = 0, Ag = 0;
  for (int i = 0; i < n_size; ++i) {
    const double d2 = wt[i] * dd[i] * dd[i];
    A2 += d2;
    Aext += d2 * q4[4 * i + 0];
    Asca += d2 * q4[4 * i + 1];
    Ag += d2 * q4[4 * i + 2];
  }
  q3[0] = Aext / A2;
  q3[1] = Asca / Aext;
  q3[2] = Ag / Asca;
}

cudaError_t mie_table_device(double m_re, double m_im, double wavelength, double d_m,
                             double sigma, int n_size, int n_angle, double* d_theta, double* d_p,
                             double* d_q3, cudaStream_t st, void* (*alloc)(size_t, void*),
                             void (*dealloc)(void*, void*), void* user) {
  if (sigma == 0.0) n_size = 1;
  // Every size parameter is below x_hi = pi d_m e^(6 sigma) / lambda, so the
  // per-size arrays are sized for its series length.
  const double pi = 3.14159265358979323846;
  const double x_hi = pi * d_m * exp(6.0 * sigma) / wavelength;
  const int nmax_hi = mie_nmax(x_hi * (1.0 + 1e-12)) + 1;
  const long long ab_stride = 2ll * (nmax_hi + 2);
  const long long d_stride = nmax_hi + 2;
  size_t sizes[8] = {
      sizeof(double) * (size_t)n_size,                       // xs
      sizeof(double) * (size_t)n_size,                       // wt
      sizeof(double) * (size_t)n_size,                       // dd
      sizeof(double) * 4 * (size_t)n_size,                   // q4
      sizeof(Cplx) * (size_t)ab_stride * n_size,             // ab
      sizeof(Cplx) * (size_t)d_stride * n_size,              // D
      sizeof(double) * (size_t)n_size * n_angle,             // out
      0};
  size_t bytes = 0;
  for (int k = 0; k < 7; ++k) bytes += (sizes[k] + 255) & ~(size_t)255;
  char* base = (char*)alloc(bytes, user);
  if (!base) return cudaErrorMemoryAllocation;
  char* ptrs[7];
  {
    char* p = base;
    for (int k = 0; k < 7; ++k) {
      ptrs[k] = p;
      p += (sizes[k] + 255) & ~(size_t)255;
    }
  }
  double* xs = (double*)ptrs[0];
  double* wt = (double*)ptrs[1];
  double* dd = (double*)ptrs[2];
  double* q4 = (double*)ptrs[3];
  Cplx* ab = (Cplx*)ptrs[4];
  Cplx* dw = (Cplx*)ptrs[5];
  double* out = (double*)ptrs[6];
  k_mie_nodes<<<(n_size + 63) / 64, 64, 0, st>>>(n_size, d_m, sigma, wavelength, xs, wt, dd);
  k_mie_coeffs<<<(n_size + 31) / 32, 32, 0, st>>>(n_size, m_re, m_im, xs, ab_stride, ab,
                                                  d_stride, dw, q4);
  dim3 g((n_angle + 127) / 128, n_size);
  k_mie_angles<<<g, 128, 0, st>>>(n_size, n_angle, xs, wt, ab_stride, ab, wavelength, out);
  k_mie_reduce<<<(n_angle + 255) / 256, 256, 0, st>>>(n_size, n_angle, out, d_theta, d_p);
  k_mie_scalars<<<1, 1, 0, st>>>(n_size, wt, dd, q4, d_q3);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  dealloc(base, user);
  return err;
}

}  // namespace pdv
