/*
 * pdv_oracle.c — plain FP64 CPU oracle for the Monte Carlo PDV spectrum
 * (Shi et al., arXiv:2012.00963, Section II).
 *
 * TEST INFRASTRUCTURE: loaded only by the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg. It shares no code with the CUDA
 * library. Slow and obvious on purpose: one packet at a time, one snapshot at
 * a time, FP64 everywhere, exact inversion of the cumulative optical depth.
 *
 * The Monte Carlo follows the paper's procedure (Section II.B, steps (1)-(7))
 * with these readings, each stated where it is used:
 *   - free paths are drawn by exact inversion of the Beer–Lambert law (Eq. 7,
 *     Eq. 10) instead of the paper's 1000-layer Bernoulli stepping (its
 *     continuum limit);
 *   - the scattering angle is drawn from the tabulated phase function by an
 *     integer inverse CDF instead of acceptance–rejection;
 *   - the apparent velocity is v_app = 1/2 sum_k (u_z,out - u_z,in) v_k over
 *     particle scatterings and free-surface reflections (Eq. 4 and Eq. 18 with
 *     the sign that makes an approaching scatterer blueshift);
 *   - the spectrum counts escaping packets by apparent velocity (Eq. 19);
 *   - optionally (implicit_capture) the absorption choice of Eq. 11 is
 *     replaced by weight reduction with Russian roulette.
 * With n_layers > 0 the paper's own scheme runs instead (orc_transport_stepped:
 * steps of H / n_layers with a Bernoulli pass per layer, acceptance-rejection
 * angles), with the readings stated there.
 */
#define _GNU_SOURCE
#include "pdv_oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_TWO32 4294967296.0

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11). Ten rounds of the 4x32 Philox S-box with the    */
/* published multipliers and Weyl key increments.                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod1;
    uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in (0, 1) from the top 23 bits: ((r >> 9) + 1/2) 2^-23, exact in
 * both binary32 and binary64 (the paper only asks for a number in (0,1),
 * Section II.B step (3)). */
static double orc_u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* 24-bit integer used for the discrete decisions (albedo test, phase bin). */
static uint32_t orc_m24(uint32_t r) { return r >> 8; }

/* ------------------------------------------------------------------------ */
/* Velocity profile and cloud constants (Eq. 8-10, Eq. 20-21, z = v t).     */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem* pb;
  double tau_tot, v_bot, v_top, d_s;
  double exp_E;          /* 1 - exp(-beta (v_top/v_fs - 1)) */
  double* M;             /* tabulated: cumulative trapezoid mass at prof_v */
  double M_tot;
  double cos_alpha;
  int cone_all, ap_all;
  uint32_t omega_q;      /* round(albedo 2^24) */
  uint64_t R_q;          /* round(R 2^32) */
  uint32_t* cq;          /* phase CDF, 2^24 scale */
  uint32_t max_events;
  double p_max;          /* largest tabulated p(theta) (acceptance-rejection) */
} orc_setup;

static int orc_setup_profile(orc_setup* st, const orc_problem* pb) {
  st->pb = pb;
  st->M = NULL;
  if (!(pb->v_fs > 0.0)) return -1;
  if (pb->profile_kind == 0) {
    if (!(pb->beta > 0.0)) return -1;
    st->v_bot = pb->v_fs;
    /* Reading: Eq. 20 runs to infinity; it is truncated where the mass tail
     * drops below 1e-6 unless v_max is given, and renormalised. */
    st->v_top = pb->v_max > 0.0 ? pb->v_max : pb->v_fs * (1.0 + log(1.0e6) / pb->beta);
    if (!(st->v_top > st->v_bot)) return -1;
    st->exp_E = -expm1(-pb->beta * (st->v_top / pb->v_fs - 1.0));
  } else if (pb->profile_kind == 1) {
    int n = pb->prof_n;
    if (n < 2 || !pb->prof_v || !pb->prof_f) return -1;
    for (int i = 0; i < n; ++i) {
      if (!(pb->prof_f[i] > 0.0)) return -1;
      if (i > 0 && !(pb->prof_v[i] > pb->prof_v[i - 1])) return -1;
    }
    if (!(pb->prof_v[0] >= pb->v_fs)) return -1;
    st->v_bot = pb->prof_v[0];
    st->v_top = pb->prof_v[n - 1];
    st->M = (double*)malloc(sizeof(double) * (size_t)n);
    st->M[0] = 0.0;
    for (int i = 0; i + 1 < n; ++i)
      st->M[i + 1] = st->M[i] + 0.5 * (pb->prof_f[i] + pb->prof_f[i + 1]) *
                                    (pb->prof_v[i + 1] - pb->prof_v[i]);
    st->M_tot = st->M[n - 1];
  } else {
    return -1;
  }
  return 0;
}

/* s(v): cumulative mass fraction between the bottom of the cloud and v. */
static double orc_cdf(const orc_setup* st, double v) {
  const orc_problem* pb = st->pb;
  if (v <= st->v_bot) return 0.0;
  if (v >= st->v_top) return 1.0;
  if (pb->profile_kind == 0)
    return -expm1(-pb->beta * (v / pb->v_fs - 1.0)) / st->exp_E;
  int n = pb->prof_n, i = 0;
  while (i + 2 < n && pb->prof_v[i + 1] <= v) ++i;
  double h = pb->prof_v[i + 1] - pb->prof_v[i];
  double k = (pb->prof_f[i + 1] - pb->prof_f[i]) / h;
  double x = v - pb->prof_v[i];
  return (st->M[i] + pb->prof_f[i] * x + 0.5 * k * x * x) / st->M_tot;
}

/* v(s): exact inverse of the cumulative mass fraction. */
static double orc_inverse(const orc_setup* st, double s) {
  const orc_problem* pb = st->pb;
  if (s <= 0.0) return st->v_bot;
  if (s >= 1.0) return st->v_top;
  if (pb->profile_kind == 0)
    return pb->v_fs * (1.0 - log1p(-s * st->exp_E) / pb->beta);
  /* piecewise-linear dm/dv: the mass is quadratic on each segment */
  double m = s * st->M_tot;
  int n = pb->prof_n, lo = 0, hi = n - 2;
  while (lo < hi) {                       /* largest i <= n-2 with M[i] <= m */
    int mid = (lo + hi + 1) / 2;
    if (st->M[mid] <= m) lo = mid; else hi = mid - 1;
  }
  int i = lo;
  double h = pb->prof_v[i + 1] - pb->prof_v[i];
  double f0 = pb->prof_f[i];
  double k = (pb->prof_f[i + 1] - f0) / h;
  double dm = m - st->M[i];
  double x = 2.0 * dm / (f0 + sqrt(f0 * f0 + 2.0 * k * dm));
  if (x > h) x = h;
  return pb->prof_v[i] + x;
}

/* normalised mass density ds/dv at v (used only for horizontal packets) */
static double orc_density(const orc_setup* st, double v) {
  const orc_problem* pb = st->pb;
  if (v < st->v_bot || v > st->v_top) return 0.0;
  if (pb->profile_kind == 0)
    return (pb->beta / pb->v_fs) * exp(-pb->beta * (v / pb->v_fs - 1.0)) / st->exp_E;
  int n = pb->prof_n, i = 0;
  while (i + 2 < n && pb->prof_v[i + 1] <= v) ++i;
  double h = pb->prof_v[i + 1] - pb->prof_v[i];
  double f = pb->prof_f[i] + (pb->prof_f[i + 1] - pb->prof_f[i]) * (v - pb->prof_v[i]) / h;
  return f / st->M_tot;
}

int orc_cloud_constants(const orc_problem* pb, double* tau_tot, double* v_bot, double* v_top,
                        double* d_sauter) {
  orc_setup st;
  memset(&st, 0, sizeof st);
  if (!(pb->rho > 0.0) || !(pb->m0 >= 0.0) || !(pb->d_m > 0.0) || !(pb->sigma_ln >= 0.0) ||
      !(pb->q_ext >= 0.0))
    return -1;
  if (orc_setup_profile(&st, pb) != 0) { free(st.M); return -1; }
  /* Sauter mean d_s = <d^3>/<d^2> of the number log-normal (Eq. 21):
   * d_m exp(2.5 sigma^2). Eq. 10 then gives the optical depth of the whole
   * cloud tau = 3 m0 Qext <d^2> / (2 rho <d^3>) = 3 m0 Qext / (2 rho d_s). */
  double d_s = pb->d_m * exp(2.5 * pb->sigma_ln * pb->sigma_ln);
  if (tau_tot) *tau_tot = 3.0 * pb->m0 * pb->q_ext / (2.0 * pb->rho * d_s);
  if (v_bot) *v_bot = st.v_bot;
  if (v_top) *v_top = st.v_top;
  if (d_sauter) *d_sauter = d_s;
  free(st.M);
  return 0;
}

double orc_profile_cdf(const orc_problem* pb, double v) {
  orc_setup st;
  memset(&st, 0, sizeof st);
  if (orc_setup_profile(&st, pb) != 0) { free(st.M); return NAN; }
  double s = orc_cdf(&st, v);
  free(st.M);
  return s;
}

double orc_profile_inverse(const orc_problem* pb, double s) {
  orc_setup st;
  memset(&st, 0, sizeof st);
  if (orc_setup_profile(&st, pb) != 0) { free(st.M); return NAN; }
  double v = orc_inverse(&st, s);
  free(st.M);
  return v;
}

/* ------------------------------------------------------------------------ */
/* Mie theory (Eq. 12-14), written from the series of Bohren & Huffman,    */
/* "Absorption and Scattering of Light by Small Particles" (1983), ch. 4:   */
/* logarithmic derivative D_n(mx) by downward recurrence, Riccati–Bessel    */
/* functions by upward recurrence, angular functions pi_n and tau_n.        */
/* The paper's Eq. 14 is garbled; S1 and S2 below are the standard ones.   */
/* ------------------------------------------------------------------------ */
int orc_mie_single(double x, double mr, double mi, int n_mu, const double* mu, double* s11,
                   double* s22, double* q, double* s0) {
  double complex m = mr + mi * I;
  double complex mx = m * x;
  int nmax = (int)floor(x + 4.0 * cbrt(x) + 2.0);  /* Wiscombe's stopping rule */
  if (nmax < 1) nmax = 1;
  int nstart = (int)ceil(cabs(mx));
  if (nstart < nmax) nstart = nmax;
  nstart += 16;
  double complex* D = (double complex*)malloc(sizeof(double complex) * (size_t)(nstart + 1));
  double complex* a = (double complex*)malloc(sizeof(double complex) * (size_t)(nmax + 2));
  double complex* b = (double complex*)malloc(sizeof(double complex) * (size_t)(nmax + 2));
  D[nstart] = 0.0;
  for (int n = nstart; n >= 1; --n) D[n - 1] = (double)n / mx - 1.0 / (D[n] + (double)n / mx);

  double psi_prev = cos(x), psi = sin(x);   /* psi_{-1}, psi_0 */
  double chi_prev = -sin(x), chi = cos(x);  /* chi_{-1}, chi_0 */
  double complex xi = psi - I * chi;        /* xi_0 */
  for (int n = 1; n <= nmax; ++n) {
    double psi_n = (2.0 * n - 1.0) / x * psi - psi_prev;
    double chi_n = (2.0 * n - 1.0) / x * chi - chi_prev;
    double complex xi_n = psi_n - I * chi_n;
    double complex da = D[n] / m + (double)n / x;
    double complex db = m * D[n] + (double)n / x;
    a[n] = (da * psi_n - psi) / (da * xi_n - xi);
    b[n] = (db * psi_n - psi) / (db * xi_n - xi);
    psi_prev = psi; psi = psi_n;
    chi_prev = chi; chi = chi_n;
    xi = xi_n;
  }
  a[nmax + 1] = 0.0;
  b[nmax + 1] = 0.0;

  double sext = 0.0, ssca = 0.0, gsum = 0.0;
  double complex sback = 0.0, sfwd = 0.0;
  for (int n = 1; n <= nmax; ++n) {
    double fn = 2.0 * n + 1.0;
    sext += fn * creal(a[n] + b[n]);
    ssca += fn * (creal(a[n]) * creal(a[n]) + cimag(a[n]) * cimag(a[n]) +
                  creal(b[n]) * creal(b[n]) + cimag(b[n]) * cimag(b[n]));
    sback += fn * ((n % 2) ? -1.0 : 1.0) * (a[n] - b[n]);
    sfwd += 0.5 * fn * (a[n] + b[n]);
    gsum += (double)n * (n + 2.0) / (n + 1.0) *
                creal(a[n] * conj(a[n + 1]) + b[n] * conj(b[n + 1])) +
            fn / ((double)n * (n + 1.0)) * creal(a[n] * conj(b[n]));
  }
  double qext = 2.0 / (x * x) * sext;
  double qsca = 2.0 / (x * x) * ssca;
  double qback = creal(sback * conj(sback)) / (x * x);
  double g = 4.0 / (x * x * qsca) * gsum;
  if (q) { q[0] = qext; q[1] = qsca; q[2] = qback; q[3] = g; }
  if (s0) { s0[0] = creal(sfwd); s0[1] = cimag(sfwd); }

  for (int j = 0; j < n_mu; ++j) {
    double u = mu[j];
    double pi_prev = 0.0, pi_n = 1.0;       /* pi_0, pi_1 */
    double complex S1 = 0.0, S2 = 0.0;
    for (int n = 1; n <= nmax; ++n) {
      double tau_n = n * u * pi_n - (n + 1.0) * pi_prev;
      double fn = (2.0 * n + 1.0) / ((double)n * (n + 1.0));
      S1 += fn * (a[n] * pi_n + b[n] * tau_n);
      S2 += fn * (a[n] * tau_n + b[n] * pi_n);
      double pi_next = ((2.0 * n + 1.0) / n) * u * pi_n - ((n + 1.0) / n) * pi_prev;
      pi_prev = pi_n;
      pi_n = pi_next;
    }
    s11[j] = creal(S1 * conj(S1));
    s22[j] = creal(S2 * conj(S2));
  }
  free(D); free(a); free(b);
  return nmax;
}

/* Gauss–Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static void orc_gauss_legendre(int n, double* z, double* w) {
  for (int i = 0; i < n; ++i) {
    double r = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = r;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      double pn = (n == 1) ? r : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (r * pn - pm) / (r * r - 1.0);
      double dr = pn / dp;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    z[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dp * dp);
  }
}

/* Size average over the number log-normal of Eq. 21, Gauss–Legendre in
 * y = ln d over [ln d_m - 6 sigma, ln d_m + 6 sigma] (the paper does not say
 * how it averages). p(theta) is proportional to <C_sca p_d(theta)> =
 * lambda^2/(8 pi^2) <|S1|^2 + |S2|^2>; albedo = <C_sca>/<C_ext>;
 * q_ext = <d^2 Q_ext>/<d^2>; g = <C_sca g>/<C_sca>. */
int orc_mie_table(double mr, double mi, double wavelength, double d_m, double sigma_ln,
                  int n_size, int n_angle, double* theta, double* p, double* q_ext,
                  double* albedo, double* g) {
  if (!(wavelength > 0.0) || !(d_m > 0.0) || !(sigma_ln >= 0.0) || n_angle < 2) return -1;
  if (sigma_ln == 0.0) n_size = 1;
  if (n_size < 1) return -1;
  double* z = (double*)malloc(sizeof(double) * (size_t)n_size);
  double* w = (double*)malloc(sizeof(double) * (size_t)n_size);
  double* mu = (double*)malloc(sizeof(double) * (size_t)n_angle);
  double* s11 = (double*)malloc(sizeof(double) * (size_t)n_angle);
  double* s22 = (double*)malloc(sizeof(double) * (size_t)n_angle);
  if (n_size == 1) { z[0] = 0.0; w[0] = 1.0; }
  else orc_gauss_legendre(n_size, z, w);
  for (int j = 0; j < n_angle; ++j) {
    theta[j] = ORC_PI * (double)j / (double)(n_angle - 1);
    mu[j] = cos(theta[j]);
    p[j] = 0.0;
  }
  double A2 = 0.0, Aext = 0.0, Asca = 0.0, Ag = 0.0;
  double half = 6.0 * sigma_ln, c = log(d_m);
  for (int i = 0; i < n_size; ++i) {
    double y, wt;
    if (n_size == 1) { y = c; wt = 1.0; }
    else {
      y = c + half * z[i];
      double t = (y - c) / sigma_ln;
      wt = half * w[i] * exp(-0.5 * t * t) / (sqrt(2.0 * ORC_PI) * sigma_ln);
    }
    double d = exp(y);
    double x = ORC_PI * d / wavelength;
    double q[4];
    orc_mie_single(x, mr, mi, n_angle, mu, s11, s22, q, NULL);
    A2 += wt * d * d;
    Aext += wt * d * d * q[0];
    Asca += wt * d * d * q[1];
    Ag += wt * d * d * q[1] * q[3];
    double scale = wt * wavelength * wavelength / (8.0 * ORC_PI * ORC_PI);
    for (int j = 0; j < n_angle; ++j) p[j] += scale * (s11[j] + s22[j]);
  }
  if (q_ext) *q_ext = Aext / A2;
  if (albedo) *albedo = Asca / Aext;
  if (g) *g = Ag / Asca;
  free(z); free(w); free(mu); free(s11); free(s22);
  return 0;
}

void orc_hg_table(double g, int n, double* theta, double* p) {
  for (int j = 0; j < n; ++j) {
    theta[j] = ORC_PI * (double)j / (double)(n - 1);
    double den = 1.0 + g * g - 2.0 * g * cos(theta[j]);
    p[j] = (1.0 - g * g) / (4.0 * ORC_PI * den * sqrt(den));
  }
}

/* ------------------------------------------------------------------------ */
/* Phase sampling (Eq. 13, Eq. 15): the paper draws theta by acceptance–    */
/* rejection; here by inverse CDF of the trapezoid-integrated p(theta)       */
/* sin(theta), quantised to 24 bits so that the bin choice is an integer     */
/* decision; theta is linear inside the chosen bin.                          */
/* ------------------------------------------------------------------------ */
int orc_phase_cdf(int n, const double* theta, const double* p, uint32_t* cq, double* g_tab) {
  if (n < 2) return -1;
  if (fabs(theta[0]) > 1e-12 || fabs(theta[n - 1] - ORC_PI) > 1e-12) return -1;
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  c[0] = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    if (!(theta[i + 1] > theta[i]) || !(p[i] >= 0.0) || !(p[i + 1] >= 0.0)) { free(c); return -1; }
    c[i + 1] = c[i] + 0.5 * (p[i] * sin(theta[i]) + p[i + 1] * sin(theta[i + 1])) *
                          (theta[i + 1] - theta[i]);
  }
  double total = c[n - 1];
  if (!(total > 0.0)) { free(c); return -1; }
  for (int i = 0; i < n; ++i) cq[i] = (uint32_t)floor(c[i] / total * 16777216.0 + 0.5);
  cq[0] = 0;
  cq[n - 1] = 16777216u;
  double gt = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    double dc = (double)(cq[i + 1] - cq[i]) / 16777216.0;
    gt += dc * (sin(theta[i + 1]) - sin(theta[i])) / (theta[i + 1] - theta[i]);
  }
  if (g_tab) *g_tab = gt;
  free(c);
  return 0;
}

double orc_phase_sample(int n, const double* theta, const uint32_t* cq, uint32_t m) {
  int lo = 0, hi = n - 2;                /* largest i <= n-2 with cq[i] <= m */
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (cq[mid] <= m) lo = mid; else hi = mid - 1;
  }
  double frac = ((double)(m - cq[lo]) + 0.5) / (double)(cq[lo + 1] - cq[lo]);
  return theta[lo] + frac * (theta[lo + 1] - theta[lo]);
}

/* Eq. 16 (standard form; the printed Eq. 16 has typos in its u_x and u_y
 * rows), with the horizontal norm s = sqrt(u_x^2 + u_y^2) taken from the
 * horizontal components, and Eq. 17 for a vertical direction. The paper says
 * only "u_z close to 1" for Eq. 17; it is read as vertical to within
 * s < 1e-15: a wider threshold makes the new direction jump (by up to
 * sqrt(2 (1 - |u_z|)) at the switch), and walks whose u_z is rounded to one
 * side of it or the other would part there. The result is renormalised. */
void orc_rotate(double u[3], double ct, double st, double cp, double sp) {
  double ux = u[0], uy = u[1], uz = u[2], nx, ny, nz;
  double h2 = ux * ux + uy * uy;
  if (h2 < 1e-30) {
    nx = st * cp;
    ny = st * sp;
    nz = uz >= 0.0 ? ct : -ct;
  } else {
    double s = sqrt(h2);
    nx = st * (ux * uz * cp - uy * sp) / s + ux * ct;
    ny = st * (uy * uz * cp + ux * sp) / s + uy * ct;
    nz = -st * cp * s + uz * ct;
  }
  double norm = sqrt(nx * nx + ny * ny + nz * nz);
  u[0] = nx / norm; u[1] = ny / norm; u[2] = nz / norm;
}

/* ------------------------------------------------------------------------ */
/* Transport of one packet at one snapshot time.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t* hist;        /* [n_bins] for this snapshot */
  uint64_t* cnt;         /* [ORC_NCOUNTERS] */
  uint64_t* order;       /* [ORC_NORDER][n_bins] or NULL */
} orc_tally;

typedef struct {
  uint32_t n_events, n_scatters, n_surface, fate;
  uint64_t weight;
  double v_app;
  int detected;
} orc_result;

static void orc_trace_put(orc_vertex* tr, int max_v, int* nv, double x, double y, double z,
                          double v, const double u[3], int kind) {
  if (!tr || *nv >= max_v) return;
  orc_vertex* e = &tr[*nv];
  e->x = x; e->y = y; e->z = z; e->v = v;
  e->ux = u[0]; e->uy = u[1]; e->uz = u[2];
  e->kind = kind;
  ++*nv;
}

/* ------------------------------------------------------------------------ */
/* Rounding sensitivity of a packet's apparent velocity (test support).       */
/* A binary32 walk rounds every flight's optical length and every new         */
/* direction, and stores each direction component to 24 bits. Re-running the  */
/* packet in FP64 with random errors of those sizes injected at those points  */
/* (stochastic arithmetic in the manner of Vignes' CESTAC method) shows how    */
/* far such roundings move v_app, whatever amplifies them: a steep dv/dS in    */
/* the thin top of the cloud, or a near-vertical direction whose azimuth      */
/* frame (Eq. 16) or Eq. 17 switch turns a 1e-7 error into a large one. The    */
/* errors are drawn from Philox under a key of their own, so the walk's own    */
/* random numbers (and with them its decisions) are unchanged.                */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t run;          /* 1, 2, ...: which perturbed re-run               */
  double sd_flight, sd_turn, sd_store;   /* already scaled by 2^-24          */
} orc_pert;

/* standard normal from two 24-bit uniforms (Box–Muller) */
static double orc_gauss(uint32_t a, uint32_t b) {
  double u1 = ((double)(a >> 8) + 0.5) / 16777216.0;
  double u2 = ((double)(b >> 8) + 0.5) / 16777216.0;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
}

/* two standard normals for (packet, event, slot) of re-run pe->run */
static void orc_pert_normals(const orc_problem* pb, const orc_pert* pe, uint64_t pk, uint32_t k,
                             uint32_t slot, double g[2]) {
  uint32_t key[2] = {(uint32_t)pb->seed ^ 0x3C6EF372u,
                     (uint32_t)(pb->seed >> 32) ^ (0x85EBCA6Bu * pe->run)};
  uint32_t ctr[4] = {(uint32_t)pk, (uint32_t)(pk >> 32), k, slot};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  g[0] = orc_gauss(r[0], r[1]);
  g[1] = orc_gauss(r[2], r[3]);
}

/* relative error factor of flight k's optical length */
static double orc_pert_flight(const orc_problem* pb, const orc_pert* pe, uint64_t pk, uint32_t k) {
  double g[2];
  orc_pert_normals(pb, pe, pk, k, 0u, g);
  return 1.0 + pe->sd_flight * g[0];
}

/* the new direction of event k as a binary32 walk would hold it: a fresh
 * error on each component, renormalised, then each component stored */
static void orc_pert_turn(const orc_problem* pb, const orc_pert* pe, uint64_t pk, uint32_t k,
                          double u[3]) {
  double a[2], b[2], c[2];
  orc_pert_normals(pb, pe, pk, k, 1u, a);
  orc_pert_normals(pb, pe, pk, k, 2u, b);
  orc_pert_normals(pb, pe, pk, k, 3u, c);
  if (pe->sd_turn != 0.0) {
    u[0] += pe->sd_turn * a[0];
    u[1] += pe->sd_turn * a[1];
    u[2] += pe->sd_turn * b[0];
    double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] /= n;
    u[1] /= n;
    u[2] /= n;
  }
  u[0] *= 1.0 + pe->sd_store * b[1];
  u[1] *= 1.0 + pe->sd_store * c[0];
  u[2] *= 1.0 + pe->sd_store * c[1];
}

/* Step (6) at the top of the cloud: vacuum flight from (x, y, z_top) to the
 * probe plane, the acceptance test, and the Eq. 19 tally. Returns detected. */
static int orc_escape(const orc_setup* st, orc_tally* ta, double x, double y, double z_top,
                      const double u[3], uint64_t W, double vapp, uint32_t order,
                      orc_vertex* trace, int max_v, int* nv) {
  const orc_problem* pb = st->pb;
  x += u[0] * (pb->z_probe - z_top) / u[2];
  y += u[1] * (pb->z_probe - z_top) / u[2];
  orc_trace_put(trace, max_v, nv, x, y, pb->z_probe, 0.0, u, 3);
  ta->cnt[ORC_ESCAPES] += 1;
  int cone_ok = st->cone_all || u[2] >= st->cos_alpha;
  int ap_ok = st->ap_all || (x * x + y * y <= pb->r_ap * pb->r_ap);
  if (!(cone_ok && ap_ok)) {
    ta->cnt[ORC_W_ESC_UNDETECTED] += W;
    return 0;
  }
  /* Eq. 19: the spectrum counts out-photons by frequency shift */
  ta->cnt[ORC_DETECTED] += 1;
  double fb = floor((vapp - pb->v_lo) * ((double)pb->n_bins / (pb->v_hi - pb->v_lo)));
  if (fb < 0.0) ta->cnt[ORC_W_UNDER] += W;
  else if (fb >= (double)pb->n_bins) ta->cnt[ORC_W_OVER] += W;
  else {
    int b = (int)fb;
    ta->hist[b] += W;
    ta->cnt[ORC_W_DETECTED] += W;
    if (ta->order) {
      uint32_t o = order;
      if (o >= ORC_NORDER) o = ORC_NORDER - 1;
      ta->order[(size_t)o * pb->n_bins + b] += W;
    }
  }
  return 1;
}

/* Step (6) at the free surface: reflectivity in 2^32 fixed point (rounded; the
 * paper has none), the new direction by the surface law from r[1], r[2], and
 * the Doppler shift of the moving wall. Returns 1 when no weight is left. */
static int orc_surface(const orc_setup* st, orc_tally* ta, const uint32_t r[4], double u[3],
                       uint64_t* Wp, double* vapp, const orc_pert* pe, uint64_t pk, uint32_t k) {
  const orc_problem* pb = st->pb;
  uint64_t W = *Wp;
  ta->cnt[ORC_EVENTS] += 1;
  ta->cnt[ORC_SURFACE_HITS] += 1;
  uint64_t Wn = st->R_q >= ((uint64_t)1 << 32) ? W : (W * st->R_q + ((uint64_t)1 << 31)) >> 32;
  ta->cnt[ORC_W_ABS_SURFACE] += W - Wn;
  *Wp = Wn;
  double uz_old = u[2];
  if (pb->surface_mode == 2) {
    u[2] = -u[2];                      /* specular */
  } else {
    double ct, stt;
    if (pb->surface_mode == 1) {       /* Lambertian: cos = sqrt(u) */
      double a = orc_u01(r[1]);
      ct = sqrt(a);
      stt = sqrt(1.0 - a);
    } else {
      /* the paper's ideal diffuse reflection (Section II.B): polar angle
       * uniform; measured from +z it is uniform in [0, pi/2) */
      double th = 0.5 * ORC_PI * orc_u01(r[1]);
      ct = cos(th);
      stt = sin(th);
    }
    double ph = 2.0 * ORC_PI * orc_u01(r[2]);
    u[0] = stt * cos(ph);
    u[1] = stt * sin(ph);
    u[2] = ct;
  }
  if (pe) orc_pert_turn(pb, pe, pk, k, u);
  /* the moving wall shifts the frequency like a particle at v_fs */
  *vapp += 0.5 * (u[2] - uz_old) * pb->v_fs;
  return Wn == 0;
}

static void orc_transport(const orc_setup* st, uint64_t pk, double t, orc_tally* ta,
                          orc_result* res, orc_vertex* trace, int max_v, const orc_pert* pe) {
  const orc_problem* pb = st->pb;
  uint32_t key[2] = {(uint32_t)pb->seed, (uint32_t)(pb->seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)pk, (uint32_t)(pk >> 32), 0u, pb->stream_id};
  uint32_t r[4];
  int nv = 0;

  /* Step (1): launch on the beam disk at the probe plane, moving along -z
   * towards the free surface (Eq. 6, incident direction n_0). The vacuum
   * flight down to the top of the cloud keeps x and y. Event index 0. */
  orc_philox4x32_10(ctr, key, r);
  double rad = pb->r_beam * sqrt(orc_u01(r[0]));
  double psi = 2.0 * ORC_PI * orc_u01(r[1]);
  double x = rad * cos(psi), y = rad * sin(psi);
  double u[3] = {0.0, 0.0, -1.0};
  if (pb->test_horizontal_launch) {  /* test of the horizontal-flight rule */
    u[0] = 1.0;
    u[2] = 0.0;
  }
  orc_trace_put(trace, max_v, &nv, x, y, pb->z_probe, 0.0, u, 0);
  double z = st->v_top * t;          /* particles at z = v t (vacuum flight) */
  double vcur = st->v_top;
  double T = st->tau_tot;            /* optical depth above the free surface */
  double vapp = 0.0;
  uint64_t W = (uint64_t)1 << 32;
  uint32_t nev = 0, nsca = 0, nsurf = 0, fate = 0;
  int detected = 0;
  const double z_fs = pb->v_fs * t;

  for (uint32_t k = 1; fate == 0; ++k) {
    ctr[2] = k;
    orc_philox4x32_10(ctr, key, r);
    /* Step (3): Beer–Lambert free path (Eq. 7, Eq. 10) sampled exactly. */
    double tau = -log(orc_u01(r[0]));
    double Tn, vn;
    int interact = 0;
    if (fabs(u[2]) < 1e-9) {
      /* horizontal packet: z is held, the lateral path is tau / mu(z) where
       * mu = dT/dz = tau_tot (ds/dv) / t (the paper is silent on this case) */
      double len = tau * t / (st->tau_tot * orc_density(st, vcur));
      x += u[0] * len;
      y += u[1] * len;
      Tn = T;
      vn = vcur;
      interact = 1;
    } else {
      double dT = tau * u[2];
      if (pe) dT *= orc_pert_flight(pb, pe, pk, k);
      Tn = T + dT;
      if (Tn >= st->tau_tot) {
        /* Step (6): leaves through the top */
        double z_top = st->v_top * t;
        x += u[0] * (z_top - z) / u[2];
        y += u[1] * (z_top - z) / u[2];
        detected = orc_escape(st, ta, x, y, z_top, u, W, vapp, nsca + nsurf, trace, max_v, &nv);
        fate = ORC_FATE_ESCAPED;
        break;
      } else if (Tn <= 0.0) {
        /* Step (6): reaches the free surface z_fs = v_fs t */
        x += u[0] * (z_fs - z) / u[2];
        y += u[1] * (z_fs - z) / u[2];
        z = z_fs;
        T = 0.0;
        vcur = pb->v_fs;
        ++nev;
        ++nsurf;
        if (orc_surface(st, ta, r, u, &W, &vapp, pe, pk, k)) {
          orc_trace_put(trace, max_v, &nv, x, y, z, pb->v_fs, u, 2);
          fate = ORC_FATE_ABS_SURFACE;
          break;
        }
        orc_trace_put(trace, max_v, &nv, x, y, z, pb->v_fs, u, 2);
      } else {
        vn = orc_inverse(st, Tn / st->tau_tot);
        double zn = vn * t;
        x += u[0] * (zn - z) / u[2];
        y += u[1] * (zn - z) / u[2];
        interact = 1;
      }
    }
    if (interact) {
      z = vn * t;
      T = Tn;
      vcur = vn;
      ++nev;
      ta->cnt[ORC_EVENTS] += 1;
      /* Step (4), Eq. 11: scatter with probability K_sca/K_ext (analog), or
       * always scatter carrying the fraction K_sca/K_ext of the weight
       * (implicit capture, with the roulette on the same draw r1) */
      int scatter;
      if (!pb->implicit_capture) {
        scatter = orc_m24(r[1]) < st->omega_q;
      } else {
        uint64_t Wn = (W * (uint64_t)st->omega_q + ((uint64_t)1 << 23)) >> 24;
        ta->cnt[ORC_W_ABS_PARTICLE] += W - Wn;
        W = Wn;
        scatter = 1;
        if (W < ORC_RR_W) {
          if (W > 0 && orc_m24(r[1]) < (1u << 24) / ORC_RR_M) {
            ta->cnt[ORC_W_RR_GAINED] += (ORC_RR_M - 1) * W;
            W *= ORC_RR_M;
          } else {
            ta->cnt[ORC_W_RR_DROPPED] += W;
            orc_trace_put(trace, max_v, &nv, x, y, z, vn, u, 4);
            fate = ORC_FATE_DROPPED;
            break;
          }
        }
      }
      if (scatter) {
        double th = orc_phase_sample(pb->n_phase, pb->theta, st->cq, orc_m24(r[2]));
        double ph = 2.0 * ORC_PI * orc_u01(r[3]);              /* Eq. 15 */
        double uz_old = u[2];
        orc_rotate(u, cos(th), sin(th), cos(ph), sin(ph));    /* Eq. 16-17 */
        if (pe) orc_pert_turn(pb, pe, pk, k, u);
        vapp += 0.5 * (u[2] - uz_old) * vn;                    /* Eq. 4, 18 */
        ++nsca;
        ta->cnt[ORC_SCATTERS] += 1;
        orc_trace_put(trace, max_v, &nv, x, y, z, vn, u, 1);
      } else {
        ta->cnt[ORC_W_ABS_PARTICLE] += W;
        orc_trace_put(trace, max_v, &nv, x, y, z, vn, u, 4);
        fate = ORC_FATE_ABS_PARTICLE;
        break;
      }
    }
    if (nev >= st->max_events) {
      /* guard against endless walks (the paper is silent) */
      ta->cnt[ORC_W_TRUNCATED] += W;
      ta->cnt[ORC_TRUNCATED] += 1;
      fate = ORC_FATE_TRUNCATED;
      break;
    }
  }
  res->n_events = nev;
  res->n_scatters = nsca;
  res->n_surface = nsurf;
  res->fate = fate;
  res->weight = W;
  res->v_app = vapp;
  res->detected = detected;
}

/* ------------------------------------------------------------------------ */
/* The paper's literal scheme (Section II.B steps (2)-(6)): synchronous      */
/* steps of H / n_layers, a Bernoulli pass per layer with the layer's        */
/* Beer-Lambert probability (Eq. 7, Eq. 10), and the polar angle by           */
/* acceptance-rejection (step (4)).                                           */
/* ------------------------------------------------------------------------ */

/* p(theta) linear between the tabulated nodes (Eq. 13 as tabulated). */
static double orc_phase_p(const orc_problem* pb, double th) {
  int lo = 0, hi = pb->n_phase - 2;
  while (lo < hi) {                       /* largest i <= n-2 with theta_i <= th */
    int mid = (lo + hi + 1) / 2;
    if (pb->theta[mid] <= th) lo = mid; else hi = mid - 1;
  }
  double a = pb->theta[lo], b = pb->theta[lo + 1];
  double f = (th - a) / (b - a);
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  return pb->p[lo] + (pb->p[lo + 1] - pb->p[lo]) * f;
}

/* Acceptance-rejection for the scattering angle: a direction uniform over the
 * sphere (cos theta uniform in (-1, 1)) is accepted with probability
 * p(theta) / max p. The draws come from a second Philox key, counter
 * (packet, step, attempt pair, -): words (r0, r1) and (r2, r3) are two
 * attempts. Returns cos theta. */
static double orc_ar_cos(const orc_setup* st, uint64_t pk, uint32_t step) {
  const orc_problem* pb = st->pb;
  uint32_t key[2] = {(uint32_t)pb->seed ^ 0xA4093822u, (uint32_t)(pb->seed >> 32) ^ pb->stream_id};
  uint32_t ctr[4] = {(uint32_t)pk, (uint32_t)(pk >> 32), step, 0u};
  uint32_t r[4];
  double mu = 0.0;
  for (uint32_t a = 0; a < (1u << 24); ++a) {
    ctr[3] = a;
    orc_philox4x32_10(ctr, key, r);
    for (int h = 0; h < 2; ++h) {
      mu = 2.0 * orc_u01(r[2 * h]) - 1.0;
      if (orc_u01(r[2 * h + 1]) * st->p_max < orc_phase_p(pb, acos(mu))) return mu;
    }
  }
  return mu;     /* 2^25 rejections in a row: keep the last proposal */
}

double orc_phase_ar_cos(const orc_problem* pb, uint64_t pk, uint32_t step) {
  orc_setup st;
  memset(&st, 0, sizeof st);
  st.pb = pb;
  for (int i = 0; i < pb->n_phase; ++i)
    if (pb->p[i] > st.p_max) st.p_max = pb->p[i];
  return orc_ar_cos(&st, pk, step);
}

static void orc_transport_stepped(const orc_setup* st, uint64_t pk, double t, orc_tally* ta,
                                  orc_result* res, orc_vertex* trace, int max_v,
                                  const orc_pert* pe) {
  const orc_problem* pb = st->pb;
  uint32_t key[2] = {(uint32_t)pb->seed, (uint32_t)(pb->seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)pk, (uint32_t)(pk >> 32), 0u, pb->stream_id};
  uint32_t r[4];
  int nv = 0;

  /* Step (1): launch as in the exact scheme (event 0) */
  orc_philox4x32_10(ctr, key, r);
  double rad = pb->r_beam * sqrt(orc_u01(r[0]));
  double psi = 2.0 * ORC_PI * orc_u01(r[1]);
  double x = rad * cos(psi), y = rad * sin(psi);
  double u[3] = {0.0, 0.0, -1.0};
  orc_trace_put(trace, max_v, &nv, x, y, pb->z_probe, 0.0, u, 0);
  const double z_fs = pb->v_fs * t, z_top = st->v_top * t;
  /* Step (2): every step is a thousandth (1 / n_layers) of the ejecta height */
  const double h = (z_top - z_fs) / (double)pb->n_layers;
  /* a step that ends within 1e-6 of the ejecta height of the top or of the
   * free surface reaches it: n_layers vertical steps land exactly on the
   * surface, and rounding must not decide whether they do */
  const double eps = 1e-6 * (z_top - z_fs);
  double z = z_top;
  double vapp = 0.0;
  uint64_t W = (uint64_t)1 << 32;
  uint32_t nev = 0, nsca = 0, nsurf = 0, fate = 0;
  int detected = 0;

  for (uint32_t k = 1; fate == 0; ++k) {
    ctr[2] = k;
    orc_philox4x32_10(ctr, key, r);
    /* Step (3): one step along u; the optical depth of the layer crossed is
     * the mass it holds (Eq. 10 per layer), over |u_z| for a slant path */
    double zn = z + u[2] * h;
    double zc = zn < z_fs ? z_fs : (zn > z_top ? z_top : zn);
    double dtau;
    if (fabs(u[2]) < 1e-9)
      dtau = st->tau_tot * orc_density(st, z / t) * h / t;
    else
      dtau = st->tau_tot * fabs(orc_cdf(st, zc / t) - orc_cdf(st, z / t)) / fabs(u[2]);
    if (orc_u01(r[0]) < exp(-dtau)) {
      /* passes the layer: step (5) moves it; step (6) checks the boundaries */
      if (zn >= z_top - eps) {
        x += u[0] * (z_top - z) / u[2];
        y += u[1] * (z_top - z) / u[2];
        detected = orc_escape(st, ta, x, y, z_top, u, W, vapp, nsca + nsurf, trace, max_v, &nv);
        fate = ORC_FATE_ESCAPED;
        break;
      } else if (zn <= z_fs + eps) {
        x += u[0] * (z_fs - z) / u[2];
        y += u[1] * (z_fs - z) / u[2];
        z = z_fs;
        ++nev;
        ++nsurf;
        int dead = orc_surface(st, ta, r, u, &W, &vapp, pe, pk, k);
        orc_trace_put(trace, max_v, &nv, x, y, z, pb->v_fs, u, 2);
        if (dead) {
          fate = ORC_FATE_ABS_SURFACE;
          break;
        }
      } else {
        x += u[0] * h;
        y += u[1] * h;
        z = zn;
      }
    } else {
      /* stopped in the layer: the interaction is at the end of the step
       * (inside the cloud); step (4) decides scatter or absorption (Eq. 11) */
      double len = fabs(u[2]) < 1e-9 ? h : (zc - z) / u[2];
      x += u[0] * len;
      y += u[1] * len;
      z = zc;
      double vn = z / t;
      ++nev;
      ta->cnt[ORC_EVENTS] += 1;
      if (orc_m24(r[1]) < st->omega_q) {
        double ct = orc_ar_cos(st, pk, k);
        double ph = 2.0 * ORC_PI * orc_u01(r[3]);              /* Eq. 15 */
        double uz_old = u[2];
        orc_rotate(u, ct, sqrt(1.0 - ct * ct), cos(ph), sin(ph));   /* Eq. 16-17 */
        if (pe) orc_pert_turn(pb, pe, pk, k, u);
        vapp += 0.5 * (u[2] - uz_old) * vn;                    /* Eq. 4, 18 */
        ++nsca;
        ta->cnt[ORC_SCATTERS] += 1;
        orc_trace_put(trace, max_v, &nv, x, y, z, vn, u, 1);
      } else {
        ta->cnt[ORC_W_ABS_PARTICLE] += W;
        orc_trace_put(trace, max_v, &nv, x, y, z, vn, u, 4);
        fate = ORC_FATE_ABS_PARTICLE;
        break;
      }
    }
    if (k >= st->max_events) {
      /* the step limit of this scheme (the paper is silent) */
      ta->cnt[ORC_W_TRUNCATED] += W;
      ta->cnt[ORC_TRUNCATED] += 1;
      fate = ORC_FATE_TRUNCATED;
      break;
    }
  }
  res->n_events = nev;
  res->n_scatters = nsca;
  res->n_surface = nsurf;
  res->fate = fate;
  res->weight = W;
  res->v_app = vapp;
  res->detected = detected;
}

/* ------------------------------------------------------------------------ */
/* Driver: packets split into contiguous ranges over threads; every thread  */
/* keeps private integer tallies, summed at the end (order independent).    */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_setup* st;
  uint64_t begin, end;   /* offsets into the request's packet range */
  uint64_t* hist;        /* private [n_snap][n_bins] */
  uint64_t* cnt;         /* private [n_snap][ORC_NCOUNTERS] */
  uint64_t* order;       /* private or NULL */
  orc_packet* packets;
  int n_trace, max_v;
  orc_vertex* trace;
  uint64_t* scratch_hist;  /* [n_bins], tallies of the perturbed re-runs */
  uint64_t* scratch_cnt;   /* [ORC_NCOUNTERS] */
} orc_job;

static void* orc_worker(void* arg) {
  orc_job* jb = (orc_job*)arg;
  const orc_setup* st = jb->st;
  const orc_problem* pb = st->pb;
  size_t nb = (size_t)pb->n_bins;
  for (uint64_t i = jb->begin; i < jb->end; ++i) {
    uint64_t pk = pb->packet_begin + i;
    uint64_t mask = 0;
    for (int s = 0; s < pb->n_snap; ++s) {
      orc_tally ta;
      ta.hist = jb->hist + (size_t)s * nb;
      ta.cnt = jb->cnt + (size_t)s * ORC_NCOUNTERS;
      ta.order = jb->order ? jb->order + (size_t)s * ORC_NORDER * nb : NULL;
      ta.cnt[ORC_LAUNCHED] += 1;
      orc_result res;
      orc_vertex* tr = NULL;
      if (s == 0 && jb->trace && i < (uint64_t)jb->n_trace)
        tr = jb->trace + (size_t)i * (size_t)jb->max_v;
      if (pb->n_layers)
        orc_transport_stepped(st, pk, pb->t_snap[s], &ta, &res, tr, jb->max_v, NULL);
      else
        orc_transport(st, pk, pb->t_snap[s], &ta, &res, tr, jb->max_v, NULL);
      if (res.detected && s < 64) mask |= (uint64_t)1 << s;
      if (s == 0 && jb->packets) {
        orc_packet* o = &jb->packets[i];
        o->n_events = res.n_events;
        o->n_scatters = res.n_scatters;
        o->n_surface = res.n_surface;
        o->fate = res.fate;
        o->weight = res.weight;
        o->v_app = res.v_app;
        o->v_app_spread = 0.0;
        o->n_unstable = 0;
        o->pad_ = 0;
        /* rounding sensitivity: perturbed re-runs into a scratch tally */
        for (uint32_t q = 1; q <= pb->spread_runs; ++q) {
          const double unit = 1.0 / 16777216.0;
          orc_pert pe = {q, pb->spread_flight * unit, pb->spread_turn * unit,
                         pb->spread_store * unit};
          orc_tally sc;
          memset(jb->scratch_cnt, 0, sizeof(uint64_t) * ORC_NCOUNTERS);
          sc.hist = jb->scratch_hist;
          sc.cnt = jb->scratch_cnt;
          sc.order = NULL;
          orc_result rq;
          if (pb->n_layers)
            orc_transport_stepped(st, pk, pb->t_snap[0], &sc, &rq, NULL, 0, &pe);
          else
            orc_transport(st, pk, pb->t_snap[0], &sc, &rq, NULL, 0, &pe);
          if (rq.n_events != res.n_events) {
            o->n_unstable += 1;
          } else {
            double d = fabs(rq.v_app - res.v_app);
            if (d > o->v_app_spread) o->v_app_spread = d;
          }
        }
      }
    }
    if (jb->packets) jb->packets[i].detect_mask = mask;
  }
  return NULL;
}

int orc_simulate(const orc_problem* pb, int n_threads, uint64_t* hist, uint64_t* counters,
                 uint64_t* order_hist, orc_packet* packets, int n_trace, int max_vertices,
                 orc_vertex* trace) {
  orc_setup st;
  memset(&st, 0, sizeof st);
  if (orc_cloud_constants(pb, &st.tau_tot, NULL, NULL, &st.d_s) != 0) return -1;
  if (orc_setup_profile(&st, pb) != 0) { free(st.M); return -1; }
  if (!(pb->reflectivity >= 0.0 && pb->reflectivity <= 1.0) ||
      (pb->implicit_capture && pb->n_layers > 0) ||
      (pb->test_horizontal_launch && pb->n_layers > 0) ||
      !(pb->albedo >= 0.0 && pb->albedo <= 1.0) || pb->n_bins < 1 || !(pb->v_hi > pb->v_lo) ||
      pb->n_snap < 1 || !(pb->r_beam >= 0.0) || pb->surface_mode < 0 || pb->surface_mode > 2) {
    free(st.M);
    return -1;
  }
  for (int s = 0; s < pb->n_snap; ++s)
    if (!(pb->t_snap[s] > 0.0) || !(st.v_top * pb->t_snap[s] < pb->z_probe)) { free(st.M); return -1; }
  st.cq = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)pb->n_phase);
  if (orc_phase_cdf(pb->n_phase, pb->theta, pb->p, st.cq, NULL) != 0) {
    free(st.M); free(st.cq);
    return -1;
  }
  st.cone_all = pb->cone_alpha >= 0.5 * ORC_PI;
  st.cos_alpha = cos(pb->cone_alpha);
  st.ap_all = !(pb->r_ap > 0.0);
  st.omega_q = (uint32_t)floor(pb->albedo * 16777216.0 + 0.5);
  st.R_q = (uint64_t)floor(pb->reflectivity * ORC_TWO32 + 0.5);
  st.max_events = pb->max_events ? pb->max_events : 1000000u;
  st.p_max = 0.0;
  for (int i = 0; i < pb->n_phase; ++i)
    if (pb->p[i] > st.p_max) st.p_max = pb->p[i];

  size_t nb = (size_t)pb->n_bins, ns = (size_t)pb->n_snap;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > pb->n_packets && pb->n_packets > 0) n_threads = (int)pb->n_packets;
  if (pb->n_packets == 0) n_threads = 1;
  orc_job* jobs = (orc_job*)calloc((size_t)n_threads, sizeof(orc_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int j = 0; j < n_threads; ++j) {
    orc_job* jb = &jobs[j];
    jb->st = &st;
    jb->begin = pb->n_packets * (uint64_t)j / (uint64_t)n_threads;
    jb->end = pb->n_packets * (uint64_t)(j + 1) / (uint64_t)n_threads;
    jb->hist = (uint64_t*)calloc(ns * nb, sizeof(uint64_t));
    jb->cnt = (uint64_t*)calloc(ns * ORC_NCOUNTERS, sizeof(uint64_t));
    jb->order = order_hist ? (uint64_t*)calloc(ns * ORC_NORDER * nb, sizeof(uint64_t)) : NULL;
    jb->packets = packets;
    jb->n_trace = trace ? n_trace : 0;
    jb->max_v = max_vertices;
    jb->trace = trace;
    jb->scratch_hist = (uint64_t*)calloc(nb, sizeof(uint64_t));
    jb->scratch_cnt = (uint64_t*)calloc(ORC_NCOUNTERS, sizeof(uint64_t));
  }
  if (trace)
    for (size_t i = 0; i < (size_t)n_trace * (size_t)max_vertices; ++i) trace[i].kind = -1;
  for (int j = 1; j < n_threads; ++j) pthread_create(&th[j], NULL, orc_worker, &jobs[j]);
  orc_worker(&jobs[0]);
  for (int j = 1; j < n_threads; ++j) pthread_join(th[j], NULL);

  memset(hist, 0, sizeof(uint64_t) * ns * nb);
  memset(counters, 0, sizeof(uint64_t) * ns * ORC_NCOUNTERS);
  if (order_hist) memset(order_hist, 0, sizeof(uint64_t) * ns * ORC_NORDER * nb);
  for (int j = 0; j < n_threads; ++j) {
    for (size_t i = 0; i < ns * nb; ++i) hist[i] += jobs[j].hist[i];
    for (size_t i = 0; i < ns * ORC_NCOUNTERS; ++i) counters[i] += jobs[j].cnt[i];
    if (order_hist)
      for (size_t i = 0; i < ns * ORC_NORDER * nb; ++i) order_hist[i] += jobs[j].order[i];
    free(jobs[j].hist); free(jobs[j].cnt); free(jobs[j].order);
    free(jobs[j].scratch_hist); free(jobs[j].scratch_cnt);
  }
  free(jobs); free(th); free(st.M); free(st.cq);
  return 0;
}
