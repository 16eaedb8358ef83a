// stepping.cu — the paper's own transport scheme, taken literally
// (arXiv:2012.00963 Section II.B steps (2)-(6)):
//   (2) every step is H / n_layers long (H: the ejecta height v_max t - v_fs t);
//   (3) the photon takes one step along its direction; it passes the layer it
//       crossed with the Beer-Lambert probability of the mass the layer holds
//       (Eq. 7, Eq. 10), drawn as a Bernoulli trial;
//   (4) a photon stopped in the layer interacts at the end of the step: it is
//       absorbed or scattered (Eq. 11), the polar angle by acceptance-rejection
//       against p(theta) (a direction uniform over the sphere, accepted with
//       probability p(theta) / max p), the azimuth uniform (Eq. 15), the new
//       direction by Eq. 16-17 and the Doppler update by Eq. 4 / Eq. 18;
//   (6) the free surface reflects, the top lets photons out to the probe.
//
// The photon's height is the fixed-point coordinate P = (v - v_bot) /
// (v_top - v_bot) 2^62 of the velocity variable v = z / t, so that a step is
// the same in P at every snapshot time (one history serves all of them), and
// the mass S(P) held below a height is the velocity table's interpolation in
// exact integer arithmetic; for the exponential law of Eq. 20 the layer mass
// is evaluated in closed form instead (exp(-x0) (1 - exp(-dx)) / E), so the
// layer optical depth tau_tot dS / |u_z| carries neither cancellation nor the
// table's interpolation error.
//
// Scheduling: one photon per lane, claimed one at a time. A step's decision is
// a pure function of (height, direction, step index), and nothing else
// changes while a photon passes layers (the lateral shift of a run of passed
// layers is taken when the run ends). So once a photon has passed a few
// layers in a row, the whole warp moves it on 32 steps per round, one lane
// per step, up to the step that ends the run; the photon's lane then takes
// that step itself. The histories are the ones the step-by-step loop makes,
// bit for bit, whatever the schedule, and the near-horizontal photons that
// wander high in the thin top of the cloud for up to 1e6 steps no longer
// hold the launch open one step per iteration.
//
// Random numbers: step k of packet p draws Philox4x32-10 with counter
// (p, k, stream) under the request's seed (k = 0 is the launch): word 0 the
// Bernoulli trial, word 1 scatter/absorb (24-bit) or the surface polar angle,
// word 2 the surface azimuth, word 3 the scattering azimuth. The
// acceptance-rejection draws use a second key (seed ^ 0xA4093822, seed_hi ^
// stream) and counter (p, k, attempt pair), two attempts per call. Both keys'
// ten round keys are computed once per launch and read from shared memory.
#include <cmath>

#include "stepping.cuh"

namespace pdv {

namespace {

constexpr unsigned kFullS = 0xffffffffu;
constexpr long long kOneP = 1ll << 62;

struct StepSmem {
  size_t o_sq, o_pn, o_th, o_ts, bytes;
};

__host__ __device__ inline size_t align16s(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline StepSmem step_layout(int n_v, int n_p, int n_snap, int uniform) {
  StepSmem L;
  size_t o = 0;
  L.o_sq = o; o = align16s(o + sizeof(unsigned long long) * (size_t)(n_v + 1));
  L.o_pn = o; o = align16s(o + sizeof(float) * (size_t)n_p);
  L.o_th = o; o = align16s(o + sizeof(float) * (size_t)(uniform ? 0 : n_p));
  L.o_ts = o; o = align16s(o + sizeof(float) * (size_t)n_snap);
  L.bytes = o;
  return L;
}

// S(P), 2^62 scale: 0 below the cloud, 2^62 above it, and inside the table's
// linear interpolation between its velocity nodes, in integer arithmetic.
__device__ __forceinline__ long long mass_at(const unsigned long long* Sq, int n_v, long long P) {
  if (P <= 0) return 0;
  if (P >= kOneP) return kOneP;
  const unsigned long long q = (unsigned long long)P << 2;           // P 2^2 < 2^64
  const int j = (int)__umul64hi(q, (unsigned long long)n_v);         // floor(P n_v / 2^62)
  const unsigned long long frac = q * (unsigned long long)n_v;       // position in the node, 2^64 scale
  const unsigned long long s0 = PDV_LD(Sq, j, n_v + 1, PDV_DEBUG_SITE_MASS_NODE);
  const unsigned long long s1 = PDV_LD(Sq, j + 1, n_v + 1, PDV_DEBUG_SITE_MASS_NODE);
  return (long long)(s0 + __umul64hi(s1 - s0, frac));
}

// p(theta) / max p at cos(theta) = mu, linear in theta between the nodes.
__device__ __forceinline__ float phase_ratio(float mu, const float* pn, const float* thpi, int n_p,
                                             int uniform, float inv_nm1) {
  const float tpi = acosf(mu) * 0.318309886183790672f;               // theta / pi
  int i;
  float f;
  if (uniform) {
    const float pos = tpi / inv_nm1;
    i = min((int)pos, n_p - 2);
    f = pos - (float)i;
  } else {
    int lo = 0, hi = n_p - 2;                                         // largest thpi_i <= tpi
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (PDV_LD(thpi, mid, n_p, PDV_DEBUG_SITE_PHASE_NODE) <= tpi) lo = mid; else hi = mid - 1;
    }
    i = lo;
    const float t0 = PDV_LD(thpi, i, n_p, PDV_DEBUG_SITE_PHASE_NODE);
    f = (tpi - t0) / (PDV_LD(thpi, i + 1, n_p, PDV_DEBUG_SITE_PHASE_NODE) - t0);
  }
  f = fminf(fmaxf(f, 0.0f), 1.0f);
  const float p0 = PDV_LD(pn, i, n_p, PDV_DEBUG_SITE_PHASE_NODE);
  return fmaf(PDV_LD(pn, i + 1, n_p, PDV_DEBUG_SITE_PHASE_NODE) - p0, f, p0);
}

// Section II.B step (4): acceptance-rejection for cos(theta), run by the whole
// warp for one lane's packet. Attempt pairs are independent Philox counters,
// so lane i tries pair base + i; the first acceptance in counter order (lowest
// lane, then the pair's first attempt) is the one a sequential loop would take.
__device__ __forceinline__ float ar_cos_warp(unsigned long long pk, unsigned step, const uint2* rk2,
                                             const float* pn, const float* thpi, int n_p,
                                             int uniform, float inv_nm1, int lane) {
  float last = 0.0f;
  for (unsigned base = 0; base < (1u << 24); base += 32) {
    const uint4 r = philox4x32_10_rk(
        make_uint4((unsigned)pk, (unsigned)(pk >> 32), step, base + (unsigned)lane), rk2);
    const float mu0 = fmaf(2.0f, u23f(r.x), -1.0f);                   // exact
    const float mu1 = fmaf(2.0f, u23f(r.z), -1.0f);
    const bool acc0 = u23f(r.y) < phase_ratio(mu0, pn, thpi, n_p, uniform, inv_nm1);
    const bool acc1 = u23f(r.w) < phase_ratio(mu1, pn, thpi, n_p, uniform, inv_nm1);
    const unsigned b = __ballot_sync(kFullS, acc0 || acc1);
    if (b) return __shfl_sync(kFullS, acc0 ? mu0 : mu1, __ffs(b) - 1);
    last = __shfl_sync(kFullS, mu1, 31);
  }
  return last;     // 2^25 rejections in a row: the last proposal
}

// Height in m/s above v_bot from the fixed-point coordinate, through a 32-bit
// conversion (P >> 32 keeps 30 significant bits; 64-bit integer conversions
// run on the narrow FP64 pipe of this GPU).
__device__ __forceinline__ float p_to_v(long long P, float v_per_P32) {
  return (float)(int)(P >> 32) * v_per_P32;
}

// |u_z| h_P in P units: u_z to 32-bit fixed point, then the high half of a
// 64 x 64 product (2^-32 relative, no 64-bit conversion).
__device__ __forceinline__ long long step_P(float uz, unsigned long long h_P) {
  const unsigned m = __float2uint_rz(fabsf(uz) * 4294967296.0f);    // saturates at |u_z| = 1
  const long long d = (long long)__umul64hi((unsigned long long)m << 32, h_P);
  return uz < 0.0f ? -d : d;
}

// exp(y) - 1: the Taylor series through y^6 for |y| <= 1/16 (truncation below
// 2e-11 relative, i.e. exact at binary32), the library function beyond.
__device__ __forceinline__ float expm1_small(float y) {
  if (fabsf(y) > 0.0625f) return expm1f(y);
  const float p = fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 1.0f / 720.0f, 1.0f / 120.0f),
                                                1.0f / 24.0f), 1.0f / 6.0f), 0.5f), 1.0f);
  return y * p;
}

__device__ __forceinline__ void launch_xy(unsigned long long pk, unsigned sid, uint2 key,
                                          float r_beam, float& x0, float& y0) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)pk, (unsigned)(pk >> 32), 0u, sid), key);
  const float rad = r_beam * sqrtf(u23f(r.x));
  float sp, cp;
  sincospif(2.0f * u23f(r.y), &sp, &cp);
  x0 = rad * cp;
  y0 = rad * sp;
}

__device__ __forceinline__ void kahan(float& sum, float& comp, float term) {
  const float y = term - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// What a step depends on through the direction alone: its length in P, the
// layer term exp(-dx) - 1 of an unclipped step (Eq. 20 closed form), and
// 1 / |u_z|. Taken once per direction; both the per-lane loop and the warp's
// fast-forward read the same values.
struct StepDir {
  long long dP;            // signed step in P
  float em1;               // exp(-dx) - 1 for a step of dP (exponential law)
  float iauz;              // 1 / |u_z| (unused for a horizontal photon)
};

__device__ __forceinline__ StepDir step_dir(const StepConst& sc, float vPd, float uz) {
  StepDir d;
  d.dP = step_P(uz, (unsigned long long)sc.h_P);
  d.em1 = sc.expo ? expm1_small(-(sc.b_vfs * ((float)(int)(d.dP >> sc.shift_d) * vPd))) : 0.0f;
  d.iauz = 1.0f / fabsf(uz);
  return d;
}

// Section II.B steps (2)-(3) for one step of a photon at height P moving with
// u_z: the step's end Pn, that end inside the cloud Pc, and whether the photon
// passes the layer it crossed (the Bernoulli trial on word rx of its draw).
// A pure function of (P, direction, rx), so the per-lane loop and the warp's
// fast-forward below take identical decisions from it. `clip` says whether a
// step clipped at the cloud's ends takes its own layer term (the per-lane
// loop); the fast-forward skips that, since a clipped step ends the run
// whatever its trial gives.
template <bool CLIP>
__device__ __forceinline__ bool step_passes(const StepConst& sc, const unsigned long long* Sq,
                                            int n_v, float vP32, float vPd, long long P, float uz,
                                            const StepDir& dir, unsigned rx, long long& Pn,
                                            long long& Pc) {
  Pn = P + dir.dP;
  Pc = Pn < sc.P_fs ? sc.P_fs : (Pn > kOneP ? kOneP : Pn);
  const bool horizontal = fabsf(uz) < 1e-9f;
  float dtau;
  if (sc.expo) {
    // Eq. 20 in closed form: with x = beta (v - v_fs) / v_fs the mass
    // fraction between two heights is exp(-x0) (1 - exp(-(x1 - x0))) / E
    const float e0 = expf(-sc.b_vfs * p_to_v(P, vP32));
    if (horizontal) {
      dtau = sc.tau_f * sc.b_vfs * e0 * sc.invE * sc.h_v;
    } else {
      float em1 = dir.em1;
      if (CLIP && Pc != Pn)
        em1 = expm1_small(-(sc.b_vfs * ((float)(int)((Pc - P) >> sc.shift_d) * vPd)));
      dtau = sc.tau_f * e0 * fabsf(em1) * sc.invE * dir.iauz;
    }
  } else if (horizontal) {
    float d = 0.0f;
    if (P > 0 && P < kOneP) {
      const int j = (int)__umul64hi((unsigned long long)P << 2, (unsigned long long)n_v);
      d = u64_to_f(PDV_LD(Sq, j + 1, n_v + 1, PDV_DEBUG_SITE_MASS_NODE) -
                   PDV_LD(Sq, j, n_v + 1, PDV_DEBUG_SITE_MASS_NODE));
    }
    dtau = d * sc.tau_hv_dv;
  } else {
    const long long dS = mass_at(Sq, n_v, Pc) - mass_at(Sq, n_v, P);
    dtau = u64_to_f((unsigned long long)(dS < 0 ? -dS : dS)) * sc.tau_S * dir.iauz;
  }
  return u23f(rx) < expf(-dtau);
}

// A run of passed layers, 32 steps at a time: lane i evaluates step
// k + adv + i of one photon, and the first lane whose step would end the run
// (a stop, the top, the free surface, or a step at or past k_lim) bounds the
// advance. Every lane of the warp calls it with the same arguments; the
// result is the number of steps the photon passes before the one that ends
// its run, which the photon's own lane then takes as usual. Positions stay
// within 33 steps of the cloud: inside the 64-bit range for steps h_P <= 2^56.
__device__ __forceinline__ unsigned long long fast_forward(const StepConst& sc, const unsigned long long* Sq,
                                           int n_v, float vP32, float vPd, const uint2* rk,
                                           unsigned sid, unsigned long long pk, unsigned k,
                                           unsigned k_lim, long long P, float uz, int lane) {
  const StepDir dir = step_dir(sc, vPd, uz);
  const long long top = kOneP - sc.eps_P, bottom = sc.P_fs + sc.eps_P;
  const long long step32 = 32 * dir.dP;
  long long Pi = P + (long long)lane * dir.dP;
  unsigned long long adv = 0;
  for (;;) {
    const unsigned long long kk = (unsigned long long)k + adv + (unsigned)lane;
    bool cont = false;
    if (kk < (unsigned long long)k_lim) {
      const uint4 r = philox4x32_10_rk(
          make_uint4((unsigned)pk, (unsigned)(pk >> 32), (unsigned)kk, sid), rk);
      long long Pn, Pc;
      cont = step_passes<false>(sc, Sq, n_v, vP32, vPd, Pi, uz, dir, r.x, Pn, Pc) && Pn < top &&
             Pn > bottom;
    }
    const unsigned b = __ballot_sync(kFullS, !cont);
    if (b) return adv + (unsigned)(__ffs(b) - 1);
    adv += 32;
    Pi += step32;
  }
}

// A photon whose current run has passed this many layers is moved on by the
// whole warp (fast_forward) until the run ends.
constexpr unsigned kLongRun = 4;

// 3 blocks of 8 warps per SM (80 registers, no spills): 1.6 % faster than 2 blocks at 113
__global__ void __launch_bounds__(256, 3) k_transport_step(const SetDesc* __restrict__ set,
                                                           const float* __restrict__ pn_g,
                                                           StepConst sc,
                                                           unsigned long long* __restrict__ ctr,
                                                           unsigned long long* __restrict__ steps_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SetDesc sd;
  __shared__ unsigned long long s_cnt[C_NCOUNT];
  __shared__ unsigned long long s_steps;
  __shared__ uint2 s_rk[10], s_rk2[10];          // Philox round keys: steps, angles
  {
    const int* src = reinterpret_cast<const int*>(set);
    int* dst = reinterpret_cast<int*>(&sd);
    for (int i = threadIdx.x; i < (int)(sizeof(SetDesc) / sizeof(int)); i += blockDim.x)
      dst[i] = src[i];
    if (threadIdx.x < C_NCOUNT) s_cnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) s_steps = 0ull;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    s_rk[threadIdx.x] = philox_round_key(make_uint2((unsigned)sd.seed, (unsigned)(sd.seed >> 32)),
                                         threadIdx.x);
    s_rk2[threadIdx.x] = philox_round_key(make_uint2(sc.key2x, sc.key2y), threadIdx.x);
  }
  const StepSmem L = step_layout(sd.n_v, sd.n_p, sd.n_snap, sd.phase_uniform);
  unsigned long long* Sq = reinterpret_cast<unsigned long long*>(smem + L.o_sq);
  float* pn = reinterpret_cast<float*>(smem + L.o_pn);
  float* thpi = reinterpret_cast<float*>(smem + L.o_th);
  float* ts = reinterpret_cast<float*>(smem + L.o_ts);
  for (int i = threadIdx.x; i <= sd.n_v; i += blockDim.x) Sq[i] = sd.Sq[i];
  for (int i = threadIdx.x; i < sd.n_p; i += blockDim.x) {
    pn[i] = pn_g[i];
    if (!sd.phase_uniform) thpi[i] = sd.thpi[i];
  }
  for (int i = threadIdx.x; i < sd.n_snap; i += blockDim.x) ts[i] = (float)sd.t_snap[i];
  __syncthreads();

  const uint2 key = make_uint2((unsigned)sd.seed, (unsigned)(sd.seed >> 32));
  const unsigned sid = sd.stream_id;
  const int n_bins = sd.n_bins, row = hist_row(sd.n_bins), n_snap = sd.n_snap;
  const long long n_tally = (long long)n_snap * row;   // the debug build checks tallies against it
  (void)n_tally;
  const float vP32 = sc.v_per_P * 4294967296.0f;           // m/s per unit of P >> 32
  const float vPd = sc.v_per_P * (float)(1ll << sc.shift_d);    // m/s per unit of dP >> shift_d

  unsigned st_launch = 0, st_events = 0, st_scat = 0, st_surf = 0;
  unsigned long long st_steps = 0;
  bool alive = false;
  unsigned long long pk = 0, W = 0, dmask = 0;
  long long P = 0;
  unsigned k = 0, nev = 0, nsca = 0, nsurf = 0;
  unsigned npass = 0;          // layers passed since the last event (the current run)
  float vcur = 0.f, ux = 0.f, uy = 0.f, uz = -1.f, iuz = -1.f;
  float Xx = 0.f, Xy = 0.f, vapp = 0.f, vcomp = 0.f;

  const int lane = threadIdx.x & 31;
  bool exhausted = false;
  for (;;) {
    if (!alive && !exhausted) {
      // Step (1): the next packet of the request, at the top moving along -z
      const unsigned long long i = atomicAdd(ctr, 1ull);
      if (i >= sd.n_packets) {
        exhausted = true;
      } else {
        pk = sd.packet_begin + i;
        alive = true;
      }
      if (alive) {
        P = kOneP;
        vcur = sd.v_top_f;
        ux = 0.f; uy = 0.f; uz = -1.f; iuz = -1.f;
        Xx = 0.f; Xy = 0.f; vapp = 0.f; vcomp = 0.f;
        W = 1ull << 32;
        k = 1; nev = 0; nsca = 0; nsurf = 0; dmask = 0; npass = 0;
        ++st_launch;
      }
    }
    if (!__any_sync(kFullS, alive)) break;
    if (sc.ff) {
      // long runs of passed layers, one photon at a time by the whole warp
      unsigned todo = __ballot_sync(kFullS, alive && npass >= kLongRun);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const unsigned long long spk = __shfl_sync(kFullS, pk, src);
        const unsigned sk = __shfl_sync(kFullS, k, src);
        const long long sP = __shfl_sync(kFullS, P, src);
        const float suz = __shfl_sync(kFullS, uz, src);
        const unsigned long long adv = fast_forward(sc, Sq, sd.n_v, vP32, vPd, s_rk, sid, spk, sk,
                                                    sd.max_events, sP, suz, lane);
        if (lane == src && adv) {
          k += (unsigned)adv;
          P += (long long)adv * step_P(uz, (unsigned long long)sc.h_P);
          npass += (unsigned)adv;
          st_steps += adv;
        }
      }
    }
    unsigned fate = 0;
    bool need_ar = false;
    unsigned r_phi = 0;
    if (alive) {
      const uint4 r = philox4x32_10_rk(make_uint4((unsigned)pk, (unsigned)(pk >> 32), k, sid), s_rk);
      // Step (3): one step along u and the Bernoulli trial of the layer crossed
      long long Pn, Pc;
      const bool pass = step_passes<true>(sc, Sq, sd.n_v, vP32, vPd, P, uz,
                                          step_dir(sc, vPd, uz), r.x, Pn, Pc);
      ++st_steps;
      if (pass && Pn < kOneP - sc.eps_P && Pn > sc.P_fs + sc.eps_P) {
        P = Pn;                                           // Step (5): passed the layer
        ++npass;
      } else {
        // The run ends. Its passed layers moved the photon npass steps of
        // h along u: lateral displacement and height, taken here at once.
        if (npass) {
          const float len = (float)npass * sc.h_v;
          Xx = fmaf(ux, len, Xx);
          Xy = fmaf(uy, len, Xy);
          vcur = p_to_v(P, vP32) + sd.v_bot_f;
          npass = 0;
        }
        if (pass && Pn >= kOneP - sc.eps_P) {
          // Step (6): out through the top; vacuum flight to the probe plane
          const float d = sd.v_top_f - vcur;
          Xx = fmaf(ux * iuz, d, Xx);
          Xy = fmaf(uy * iuz, d, Xy);
          if (sd.cone_all || uz >= sd.cos_alpha_f) {
            const float fb = floorf((vapp - vcomp - sd.v_lo_f) * sd.inv_dbin_f);
            const int idx = fb < 0.0f ? 0 : (fb >= (float)n_bins ? n_bins + 1 : (int)fb + 1);
            if (sd.ap_all) {
              // every snapshot time alike: one tally in row 0 (the
              // normalisation reads it for each time)
              if (PDV_IN(idx, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
                atomicAdd(&sd.hist[idx], W);                                // Eq. 19
              if (PDV_IN(n_bins + 2, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
                atomicAdd(&sd.hist[n_bins + 2], 1ull);
              dmask = n_snap >= 64 ? ~0ull : ((1ull << n_snap) - 1ull);
            } else {
              float x0, y0;
              launch_xy(pk, sid, key, sd.r_beam_f, x0, y0);
              const float tx = ux * iuz, ty = uy * iuz;
              const float ax = fmaf(tx, sd.z_probe_f, x0), ay = fmaf(ty, sd.z_probe_f, y0);
              const float bx = fmaf(-tx, sd.v_top_f, Xx), by = fmaf(-ty, sd.v_top_f, Xy);
              for (int s = 0; s < n_snap; ++s) {
                const float t = PDV_LD(ts, s, n_snap, PDV_DEBUG_SITE_SNAPSHOT);
                const float dx = fmaf(t, bx, ax), dy = fmaf(t, by, ay);
                if (fmaf(dx, dx, dy * dy) <= sd.r_ap2_f) {
                  if (PDV_IN((long long)s * row + idx, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
                    atomicAdd(&sd.hist[(size_t)s * row + idx], W);         // Eq. 19
                  if (PDV_IN((long long)s * row + n_bins + 2, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
                    atomicAdd(&sd.hist[(size_t)s * row + n_bins + 2], 1ull);
                  if (s < 64) dmask |= 1ull << s;
                }
              }
            }
          }
          atomicAdd(&s_cnt[C_ESCAPES], 1ull);
          atomicAdd(&s_cnt[C_W_ESCAPED], W);
          fate = 1;
        } else if (pass) {
          // Step (6): the free surface; reflectivity in 2^32 fixed point
          const float d = sd.v_fs_f - vcur;
          Xx = fmaf(ux * iuz, d, Xx);
          Xy = fmaf(uy * iuz, d, Xy);
          P = sc.P_fs;
          vcur = sd.v_fs_f;
          ++nev; ++nsurf; ++st_events; ++st_surf;
          const unsigned long long Wn =
              sd.R_q >= (1ull << 32) ? W : ((W * sd.R_q + (1ull << 31)) >> 32);
          if (Wn != W) atomicAdd(&s_cnt[C_W_ABS_SURFACE], W - Wn);
          W = Wn;
          float nx, ny, nz;
          if (sd.surface_mode == PDV_SURFACE_SPECULAR) {
            nx = ux; ny = uy; nz = -uz;
          } else {
            float st, ct, sp, cp;
            if (sd.surface_mode == PDV_SURFACE_LAMBERT) {
              const float a = u23f(r.y);
              ct = sqrtf(a);
              st = sqrtf(1.0f - a);
            } else {
              sincospif(0.5f * u23f(r.y), &st, &ct);
            }
            sincospif(2.0f * u23f(r.z), &sp, &cp);
            nx = st * cp; ny = st * sp; nz = ct;
            const float inv_n = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
            nx *= inv_n; ny *= inv_n; nz *= inv_n;
          }
          kahan(vapp, vcomp, __fmul_rn(0.5f * (nz - uz), sd.v_fs_f));
          ux = nx; uy = ny; uz = nz;
          iuz = rcp_approx(nz);
          if (W == 0) fate = 3;
        } else {
          // stopped in the layer: the interaction is at the end of the step
          const float vn = Pc == sc.P_fs ? sd.v_fs_f : p_to_v(Pc, vP32) + sd.v_bot_f;
          if (fabsf(uz) < 1e-9f) {
            Xx = fmaf(ux, sc.h_v, Xx);
            Xy = fmaf(uy, sc.h_v, Xy);
          } else {
            const float d = vn - vcur;
            Xx = fmaf(ux * iuz, d, Xx);
            Xy = fmaf(uy * iuz, d, Xy);
          }
          P = Pc;
          vcur = vn;
          ++nev; ++st_events;
          if ((r.y >> 8) < sd.omega_q) {
            need_ar = true;                                               // Step (4): scattered
            r_phi = r.w;
          } else {
            atomicAdd(&s_cnt[C_W_ABS_PARTICLE], W);                       // Eq. 11: absorbed
            fate = 2;
          }
        }
      }
    }   // alive
    // the scattered lanes' polar angles, one lane at a time by the whole warp
    unsigned want = __ballot_sync(kFullS, need_ar);
    float my_ct = 0.0f;
    while (want) {
      const int src = __ffs(want) - 1;
      want &= want - 1;
      const unsigned long long spk = __shfl_sync(kFullS, pk, src);
      const unsigned sk = __shfl_sync(kFullS, k, src);
      const float c = ar_cos_warp(spk, sk, s_rk2, pn, thpi, sd.n_p, sd.phase_uniform, sd.inv_nm1,
                                  lane);
      if (lane == src) my_ct = c;
    }
    if (!alive) continue;
    if (need_ar) {
      const float ct = my_ct;
      const float st = sqrtf(fmaxf(0.0f, fmaf(-ct, ct, 1.0f)));
      float sp, cp;
      sincospif(2.0f * u23f(r_phi), &sp, &cp);                         // Eq. 15
      float nx, ny, nz;
      const float h2 = fmaf(ux, ux, uy * uy);
      if (h2 < 1e-30f) {                                             // Eq. 17: vertical
        nx = st * cp;
        ny = st * sp;
        nz = uz >= 0.0f ? ct : -ct;
      } else {                                                       // Eq. 16
        const float rs = rsqrtf(h2);
        const float s = h2 * rs;
        const float a = st * rs;
        nx = fmaf(a, fmaf(ux * uz, cp, -uy * sp), ux * ct);
        ny = fmaf(a, fmaf(uy * uz, cp, ux * sp), uy * ct);
        nz = fmaf(-st * cp, s, uz * ct);
      }
      const float inv_n = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
      nx *= inv_n; ny *= inv_n; nz *= inv_n;
      kahan(vapp, vcomp, __fmul_rn(0.5f * (nz - uz), vcur));      // Eq. 4 / Eq. 18
      ux = nx; uy = ny; uz = nz;
      iuz = rcp_approx(nz);
      ++nsca; ++st_scat;
    }
    if (fate == 0 && k >= sd.max_events) {
      atomicAdd(&s_cnt[C_W_TRUNCATED], W);
      atomicAdd(&s_cnt[C_TRUNCATED], 1ull);
      fate = 4;
    }
    ++k;
    if (fate) {
      if (sd.packets) {
        pdv_packet_record rec;
        rec.n_events = nev;
        rec.n_scatters = nsca;
        rec.n_surface = nsurf;
        rec.fate = fate;
        rec.weight = W;
        rec.v_app = (double)vapp - (double)vcomp;
        rec.detect_mask = dmask;
        if (PDV_IN(pk - sd.packet_begin, sd.n_packets, PDV_DEBUG_SITE_PACKET))
          sd.packets[pk - sd.packet_begin] = rec;
      }
      alive = false;
    }
  }

  // flush the block's counters
  atomicAdd(&s_cnt[C_LAUNCHED], (unsigned long long)st_launch);
  atomicAdd(&s_cnt[C_EVENTS], (unsigned long long)st_events);
  atomicAdd(&s_cnt[C_SCATTERS], (unsigned long long)st_scat);
  atomicAdd(&s_cnt[C_SURFACE_HITS], (unsigned long long)st_surf);
  atomicAdd(&s_steps, st_steps);
  __syncthreads();
  if (threadIdx.x < C_NCOUNT && s_cnt[threadIdx.x]) atomicAdd(&sd.cnt[threadIdx.x], s_cnt[threadIdx.x]);
  if (threadIdx.x == 0) atomicAdd(steps_out, s_steps);
}

}  // namespace

cudaError_t stepping_debug_io(DebugWord* out, bool reset, cudaStream_t st) {
#ifdef PDV_DEBUG
  return debug_word_io(out, reset, st);
#else
  (void)reset;
  (void)st;
  *out = DebugWord{};
  return cudaSuccess;
#endif
}

size_t transport_step_smem(int n_v, int n_p, int n_snap, int phase_uniform) {
  return step_layout(n_v, n_p, n_snap, phase_uniform).bytes;
}

cudaError_t transport_step_occupancy(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_transport_step,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_transport_step, 256, smem);
}

cudaError_t launch_transport_step(const SetDesc* d_set, const float* pn, const StepConst& sc,
                                  unsigned long long* d_ctr, unsigned long long* d_steps,
                                  int grid, size_t smem, cudaStream_t st) {
  k_transport_step<<<grid, 256, smem, st>>>(d_set, pn, sc, d_ctr, d_steps);
  return cudaGetLastError();
}

}  // namespace pdv
