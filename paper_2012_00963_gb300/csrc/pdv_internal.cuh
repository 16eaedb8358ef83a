// pdv_internal.cuh — device-side data layout and helpers of libpdv.
//
// The transport follows the Monte Carlo of arXiv:2012.00963 Section II:
// launch (Eq. 6), Beer–Lambert free path (Eq. 7, Eq. 10), scatter/absorb
// (Eq. 11), phase-function angle (Eq. 13-15), rotation (Eq. 16-17), Doppler
// update (Eq. 4, Eq. 18), diffuse free-surface reflection, tally (Eq. 19).
//
// Packet state on the optical-depth axis is the cumulative mass fraction
// S = T / tau_tot of the cloud below the packet (0 at the free surface, 1 at
// the top). The FP32 path holds S as a 62-bit fixed-point integer and inverts
// the velocity table with integer compares; the table itself is built in FP64.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "pdv.h"

namespace pdv {

// NVTX range for the lifetime of a scope (host code): API calls, launches,
// normalisation and the serving loop show up by name in a profiler timeline.
// Without a tool attached a push or pop is one indirect call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------- PDV_DEBUG
// The debug build checks each index into the staged tables, the tallies and
// the per-packet outputs before the access. A failed check skips the access
// and records (site, index, bound) in its translation unit's device word; the
// first failure's details are kept, later ones only counted. The release
// build compiles every check to `true`.
struct DebugWord {
  unsigned long long violations;
  long long index, bound;
  unsigned site, pad;
};

#ifdef PDV_DEBUG
constexpr bool kDebugBuild = true;
static __device__ DebugWord g_debug_word;

__device__ __noinline__ static bool debug_fail(long long i, long long n, unsigned site) {
  if (atomicAdd(&g_debug_word.violations, 1ull) == 0ull) {
    g_debug_word.index = i;
    g_debug_word.bound = n;
    g_debug_word.site = site;
  }
  return false;
}
#define PDV_IN(i, n, site)                                                          \
  ((long long)(i) >= 0 && (long long)(i) < (long long)(n)                           \
       ? true                                                                       \
       : ::pdv::debug_fail((long long)(i), (long long)(n), (site)))

// Host side: read (and optionally clear) this translation unit's word.
static inline cudaError_t debug_word_io(DebugWord* out, bool reset, cudaStream_t st) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_debug_word, sizeof(DebugWord), 0,
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && reset) {
    const DebugWord z{};
    e = cudaMemcpyToSymbolAsync(g_debug_word, &z, sizeof(DebugWord), 0, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}
#else
constexpr bool kDebugBuild = false;
#define PDV_IN(i, n, site) ((void)sizeof((i) + (n)), true)   // nothing evaluated
#endif

// Load a[i] after the check; a failed check loads a[0] (every checked table
// has at least one element).
#define PDV_LD(a, i, n, site) (PDV_IN((i), (n), (site)) ? (a)[(i)] : (a)[0])

constexpr unsigned long long kOneQ = 1ull << 62;     // S = 1 in 2^62 fixed point
constexpr double kTwo62 = 4611686018427387904.0;
constexpr double kTwo32 = 4294967296.0;
constexpr int kMaxTableNodes = 16384;
constexpr int kMaxPhase = 65536;
constexpr int kMaxSnap = 4096;
constexpr int kMaxBins = 65536;
constexpr int kGuidePhaseLog = 13;                   // 8192 guide cells over the 2^24 CDF

// Snapshot-independent counter slots of one request (device array of u64).
enum Counter {
  C_LAUNCHED = 0,
  C_EVENTS,
  C_SCATTERS,
  C_SURFACE_HITS,
  C_ESCAPES,
  C_W_ESCAPED,          // total escaped weight (split per snapshot at normalisation)
  C_W_ABS_PARTICLE,
  C_W_ABS_SURFACE,
  C_W_TRUNCATED,
  C_TRUNCATED,
  C_W_RR_DROPPED,       // weight of packets dropped by the roulette
  C_W_RR_GAINED,        // weight the roulette's survivors gained
  C_NCOUNT
};

// Per-snapshot histogram row: [under, bin 0 .. bin n-1, over, detected count].
__host__ __device__ inline int hist_row(int n_bins) { return n_bins + 3; }

// Device tables of one cloud.
struct CloudTables {
  // cumulative mass fraction at velocity nodes v_j = v_bot + j dv, j = 0..n_v
  unsigned long long* Sq = nullptr;   // [n_v + 1] S_j * 2^62 (u64)
  double* Sd = nullptr;               // [n_v + 1] S_j (FP64 path)
  float* w = nullptr;                 // [n_v] dv / (Sq_{j+1} - Sq_j)
  unsigned short* G = nullptr;        // [n_g + 1] guide: largest j <= n_v-1, Sq_j <= k 2^62 / n_g
  int n_v = 0, n_g = 0, g_shift = 0;
  // phase function
  unsigned* Cq = nullptr;             // [n_p] integer CDF, 2^24 scale
  float* thpi = nullptr;              // [n_p] theta / pi (f32)
  float* dthpi = nullptr;             // [n_p] (theta_{i+1} - theta_i) / pi / (Cq_{i+1} - Cq_i)
  double* th_d = nullptr;             // [n_p] theta (FP64 path)
  float2* cs = nullptr;               // [n_p] (cos theta_i, sin theta_i), FP64 rounded to FP32
  uint2* node = nullptr;              // [n_p] (Cq_i, slope (theta_{i+1} - theta_i) / (Cq_{i+1} - Cq_i)
                                      //  in radians as FP32 bits); slope 0 for an empty bin
  unsigned short* Gp = nullptr;       // [n_gp + 1] guide over the 2^24 CDF
  int n_p = 0;
  int phase_uniform = 0;              // theta grid uniform over [0, pi]
};

// Everything the transport needs for one request ("set"), by value.
struct SetDesc {
  const unsigned long long* Sq;
  const double* Sd;
  const float* w;
  const unsigned short* G;
  const unsigned* Cq;
  const float* thpi;
  const float* dthpi;
  const double* th_d;
  const float2* cs;                   // [n_p] (cos theta_i, sin theta_i)
  const uint2* node;                  // [n_p] (Cq_i, slope in radians per CDF unit, FP32 bits)
  const unsigned short* Gp;
  const double* t_snap;               // [3 n_snap]: seconds in request order, ascending, index
  unsigned long long* hist;           // [n_snap][n_bins + 3]
  unsigned long long* cnt;            // [C_NCOUNT]
  pdv_packet_record* packets;         // optional [n_packets]
  int n_v, n_g, g_shift, n_p;
  int n_snap, n_bins;
  int surface_mode, cone_all, ap_all, phase_uniform;   // theta_i = pi i / (n_p - 1)
  int expo;                           // exponential law (Eq. 20): velocities by its closed-form inverse
  int launch_horizontal;              // PDV_TEST_HORIZONTAL_LAUNCH: packets start along +x
  unsigned omega_q, stream_id, max_events;
  unsigned implicit;                  // PDV_IMPLICIT_CAPTURE: weight omega per interaction + roulette
  unsigned absorb_gate;               // r1 >> 8 at or above it leaves the scatter path: omega_q, or 0 (implicit)
  unsigned long long R_q, seed, packet_begin, n_packets;
  unsigned long long norm_packets;    // packets of the whole request (normalisation)
  double tau_tot, inv_tau, v_bot, dv, v_top, v_fs;
  double z_probe, r_beam, r_ap2, cos_alpha, v_lo, inv_dbin;
  float inv_tau_f, v_bot_f, dv_f, v_top_f, v_fs_f, z_probe_f, r_beam_f, r_ap2_f;
  float cos_alpha_f, v_lo_f, inv_dbin_f, inv_nm1;      // 1 / (n_p - 1)
  int angle_table;                    // node spacing <= 3.1e-3: sin/cos from the node table
  // exponential law: v(S) = v_fs - lg_c log2((1 - S) + S eps), dv/dS = dvds_c / ((1 - S) + S eps)
  float lg_c_f, eps_f, dvds_c_f;      // v_fs ln2 / beta, exp(-beta (v_top/v_fs - 1)), v_fs E / beta
  float eps30_f;                      // eps_f 2^-30 (exact): the factor of the high word of S
  double vb_d, E_d;                   // FP64 path: v_fs / beta and E = 1 - exp(-beta (v_top/v_fs - 1))
  uint2 rk[10];                       // Philox round keys of the seed (philox_round_key)
  // debug build: path trace of the first n_trace packets at snapshot time t_trace
  // (seconds), and the index check of PDV_TEST_DEBUG_CHECK
  pdv_trace_vertex* trace;
  int n_trace, max_vtx;
  double t_trace;
  int debug_check;
};

// ------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of the 4x32 S-box with the
// published multipliers and Weyl key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;   // one wide multiply
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
    c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k.x, (unsigned)p1,
                   (unsigned)(p0 >> 32) ^ c.w ^ k.y, (unsigned)p0);
  }
  return c;
}

// The same block with the ten round keys of one key read from memory (one
// shared-memory load a round in place of two additions): rk[i] is the key
// after i Weyl increments, staged once per set by philox_round_key.
__device__ __forceinline__ uint2 philox_round_key(uint2 k, unsigned i) {
  return make_uint2(k.x + i * 0x9E3779B9u, k.y + i * 0xBB67AE85u);
}

__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint2* rk) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint2 k = rk[i];
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
    c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k.x, (unsigned)p1,
                   (unsigned)(p0 >> 32) ^ c.w ^ k.y, (unsigned)p0);
  }
  return c;
}

// Uniform in (0, 1): ((r >> 9) + 1/2) 2^-23, exact in binary32 and binary64.
__device__ __forceinline__ float u23f(unsigned r) {
  return fmaf(__uint2float_rn(r >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}
__device__ __forceinline__ double u23d(unsigned r) {
  return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0);
}

// sin(pi y) and cos(pi y) for y in [0, 2] (an angle in half turns), in FP32
// with about 2 ulp error (9.1e-8 absolute): y = q/2 + r with q = rint(2 y) and
// r in [-1/4, 1/4], both exact; sin(pi r) = r P(r^2) and cos(pi r) =
// 1 + r^2 Q(r^2) by polynomials fitted here (least squares on Chebyshev
// nodes of [0, 1/4], then rounded to binary32; truncation below 1.4e-9);
// then a rotation by q quarter turns.
__device__ __forceinline__ void sincospi_half_turns(float y, float* s, float* c) {
  const float q = rintf(2.0f * y);
  const float r = fmaf(-0.5f, q, y);
  const float t = r * r;
  float p = fmaf(t, -0.5880100131034851f, 2.549651622772217f);
  p = fmaf(t, p, -5.167704105377197f);
  p = fmaf(t, p, 3.141592502593994f);
  const float sr = p * r;
  float h = fmaf(t, 0.2314641922712326f, -1.3350627422332764f);
  h = fmaf(t, h, 4.058708190917969f);
  h = fmaf(t, h, -4.934802055358887f);
  const float cr = fmaf(t, h, 1.0f);
  const int iq = (int)q & 3;
  const float a = (iq & 1) ? cr : sr, b = (iq & 1) ? sr : cr;
  *s = (iq & 2) ? -a : a;
  *c = ((iq + 1) & 2) ? -b : b;
}

// Reciprocal on the special-function unit (about 1 ulp; used for geometry
// that only feeds the lateral position).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// unsigned 64-bit integer (< 2^63) to binary32.
__device__ __forceinline__ float u64_to_f(unsigned long long d) {
  return fmaf(__uint2float_rn((unsigned)(d >> 32)), 4294967296.0f, __uint2float_rn((unsigned)d));
}

// Kernel entry points (defined in the .cu files).
// impl: some set of the launch has PDV_IMPLICIT_CAPTURE (a kernel build that
// holds the implicit-capture branch; the analog build leaves it out).
// fast: every set of the launch passes transport_fast_set (the build that
// takes those sets' branches at compile time; dumps use the generic build).
// chunk: packets a warp claims at a time (0: the default, 64)
bool transport_fast_set(const SetDesc& d);
void launch_transport_f32(const SetDesc* d_sets, int n_sets, unsigned long long* d_set_ctr,
                          int grid, int block, size_t smem, int hist_mode, bool dump, bool impl,
                          bool fast, unsigned chunk, cudaStream_t st);
// One set whose descriptor (host copy, device pointers inside) is passed by
// value as a kernel parameter.
void launch_transport_f32_one(const SetDesc& sd, unsigned long long* d_ctr, int grid, int block,
                              size_t smem, int hist_mode, bool dump, bool impl, bool fast,
                              unsigned chunk, cudaStream_t st);
void launch_transport_f64(const SetDesc* d_set, int grid, int block, cudaStream_t st);
void launch_normalise(const SetDesc* d_sets, int n_sets, double* const* d_spec,
                      pdv_counters* const* d_cnt_out, unsigned long long* const* d_raw,
                      const unsigned* flags, int max_snap, cudaStream_t st);
size_t transport_f32_smem(int n_v, int n_g, int n_p, int n_snap, int n_bins, int hist_mode,
                          int phase_uniform, int ap_all, int expo, int angle_table);
int transport_f32_max_smem();
// Load every FP32 transport build and the normalisation kernel on the current
// device now (the runtime otherwise loads a kernel at its first launch).
cudaError_t transport_preload();
cudaError_t transport_f32_occupancy(int block, size_t smem, int hist_mode, bool dump, bool impl,
                                    bool one, bool fast, int* blocks);
// The debug words of the transport and the layer-stepping translation units
// (all zero in the release build).
cudaError_t transport_debug_io(DebugWord* out, bool reset, cudaStream_t st);
cudaError_t stepping_debug_io(DebugWord* out, bool reset, cudaStream_t st);

cudaError_t build_mass_table(int kind, double beta, double v_fs, double v_bot, double v_top,
                             const double* d_prof_v, const double* d_prof_f, int prof_n,
                             double* d_prof_cum, int n_v, CloudTables* t, cudaStream_t st);
cudaError_t build_phase_cdf(const double* d_theta, const double* d_p, int n, double* d_work,
                            CloudTables* t, double* d_gtab, cudaStream_t st);
cudaError_t mie_table_device(double m_re, double m_im, double wavelength, double d_m,
                             double sigma, int n_size, int n_angle, double* d_theta, double* d_p,
                             double* d_q3, cudaStream_t st, void* (*alloc)(size_t, void*),
                             void (*dealloc)(void*, void*), void* user);

}  // namespace pdv
