// transport.cu — Monte Carlo photon-packet transport (arXiv:2012.00963,
// Section II.B steps (1)-(7)) and the tally normalisation (Eq. 19).
//
// k_transport_f32: persistent kernel. Blocks walk the list of request sets;
// for each set with packets left they stage the set's tables in shared
// memory, then every warp claims chunks of packets from the set's global
// counter and keeps its 32 lanes busy: a lane whose packet ends (escape,
// absorption, surface loss, event limit) launches the next packet of the
// warp's chunk in the same iteration. Packet state: 62-bit fixed-point mass
// fraction S (optical depth T = tau_tot S above the free surface), binary32
// direction and lateral displacement, 2^32 fixed-point weight. Histogram
// tallies are 64-bit integer atomics; the per-set sums (events, escapes,
// escaped and absorbed weight) are integers held per lane and added to the
// set's counters once per set. The set's ten Philox round keys are staged in
// shared memory with its tables. Results do not depend on scheduling.
//
// k_transport_f64: the plain FP64 path, one packet per thread at a time,
// tables read from global memory, FP64 throughout.
//
// Both kernels transport a packet once and test detection at every snapshot
// time: the cloud is self-similar (z = v t, Section II.C), so event decisions
// and the Doppler sum do not depend on t, and the lateral position at time t
// is x0 + t X with X accumulated in velocity units. With an unlimited aperture
// every time detects alike; the FP32 kernel then tallies one histogram row,
// which the normalisation reads for every time.
//
// With PDV_IMPLICIT_CAPTURE an interaction always scatters and scales the
// weight by omega in 2^32 fixed point; a packet below PDV_ROULETTE_W survives
// the roulette on the r1 draw (the analog scheme's Eq. 11 draw) with
// probability 1/16 at 16 times the weight. The roulette's rare weight sums go
// to shared atomics; the absorbed weight joins the per-lane sum.
#include <math.h>

#include "pdv_internal.cuh"

namespace pdv {

constexpr unsigned kFull = 0xffffffffu;
// Packets a warp claims from its set's counter at a time (the launch's
// chunk, pdv_tuning.tile_packets; kChunkDefault when 0)
constexpr unsigned kChunkDefault = 64;
constexpr float kTwoM62f = 2.168404344971009e-19f;   // 2^-62
constexpr float kTwoM30f = 9.313225746154785e-10f;   // 2^-30

struct SmemTables {
  const unsigned long long* Sq;
  const float* w;
  const unsigned short* G;
  const uint2* node;                  // (Cq_i, slope in radians per CDF unit) of the phase nodes
  const float* thpi;                  // coarse non-uniform tables only
  const float* dthpi;
  const unsigned short* Gp;
  const float* ts;                    // snapshot times, ascending (seconds)
  const unsigned short* perm;         // request index of each ascending time
  unsigned long long* hist;
  const float2* ang;                  // (cos, sin): the n_p phase nodes, then the kTurn turn steps
  const float2* turn;                 // ang + n_p: (cos, sin) of 2 pi j / kTurn
};

// Angles as a table value and a small remainder: cos(a + d) and sin(a + d)
// from (cos a, sin a) and cos d = 1 - d^2/2, sin d = d. For |d| <= 3.1e-3
// (half a step of the kTurn-entry table; a phase-table bin is at most 3.1e-3
// wide) the dropped terms are d^3/6 <= 5e-9 and d^4/24 <= 4e-12, below a
// binary32 ulp of a unit vector's components (6e-8).
constexpr int kTurnLog = 10, kTurn = 1 << kTurnLog;
constexpr float kPi2m25f = 9.3626757e-08f;   // pi 2^-25
constexpr float kPi2m23f = 3.7450703e-07f;   // pi 2^-23
__device__ __forceinline__ void cos_sin_add(float2 cs, float d, float* c, float* s) {
  const float cd = fmaf(d * d, -0.5f, 1.0f);
  *c = fmaf(cs.x, cd, -cs.y * d);
  *s = fmaf(cs.y, cd, cs.x * d);
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory bytes for one set's staged tables (and optional histogram).
// A uniform theta grid needs no per-node angle arrays.
// With an unlimited aperture every snapshot time detects an escaping packet
// alike, so a set tallies one histogram row (row 0) and the normalisation
// reads it for every snapshot.
__host__ __device__ inline int tally_rows(int n_snap, int ap_all) { return ap_all ? 1 : n_snap; }

__host__ __device__ inline size_t smem_layout(int n_v, int n_g, int n_p, int n_snap, int n_bins,
                                              int hist_mode, int phase_uniform, int ap_all, int expo,
                                              int angle_table, size_t* off) {
  // the exponential law inverts in closed form: its velocity table is not staged
  const size_t n_m = expo ? 0 : (size_t)n_v + 1, n_mg = expo ? 0 : (size_t)n_g + 1;
  // per-node angles in half turns: coarse tables on a non-uniform grid only
  const size_t n_th = (phase_uniform || angle_table) ? 0 : (size_t)n_p;
  size_t o = 0;
  off[0] = o; o = align16(o + sizeof(unsigned long long) * n_m);                  // Sq
  off[1] = o; o = align16(o + sizeof(float) * n_m);                               // w
  off[2] = o; o = align16(o + sizeof(unsigned short) * n_mg);                     // G
  off[3] = o; o = align16(o + sizeof(uint2) * (size_t)n_p);                       // node
  off[4] = o; o = align16(o + sizeof(float) * n_th);                              // thpi
  off[5] = o; o = align16(o + sizeof(float) * n_th);                              // dthpi
  off[6] = o; o = align16(o + sizeof(unsigned short) * ((1 << kGuidePhaseLog) + 1));  // Gp
  off[7] = o; o = align16(o + sizeof(float) * (size_t)n_snap);                    // ts
  off[8] = o; o = align16(o + sizeof(unsigned short) * (size_t)n_snap);           // perm
  off[10] = o; o = align16(o + sizeof(float2) * ((size_t)n_p + kTurn));           // ang
  off[11] = off[10] + sizeof(float2) * (size_t)n_p;                               // turn (in ang)
  off[9] = o;
  if (hist_mode == 2)
    o = align16(o + sizeof(unsigned long long) * (size_t)tally_rows(n_snap, ap_all) * hist_row(n_bins));
  return o;
}

size_t transport_f32_smem(int n_v, int n_g, int n_p, int n_snap, int n_bins, int hist_mode,
                          int phase_uniform, int ap_all, int expo, int angle_table) {
  size_t off[12];
  return smem_layout(n_v, n_g, n_p, n_snap, n_bins, hist_mode, phase_uniform, ap_all, expo,
                     angle_table, off);
}

__device__ __forceinline__ int search_mass(const unsigned long long* Sq, const unsigned short* G,
                                           int g_shift, int n_g, int n_v, unsigned long long s) {
  unsigned kg = (unsigned)(s >> g_shift);
  if (kg > (unsigned)(n_g - 1)) kg = (unsigned)(n_g - 1);
  int lo = PDV_LD(G, kg, n_g + 1, PDV_DEBUG_SITE_MASS_GUIDE);
  int hi = PDV_LD(G, kg + 1, n_g + 1, PDV_DEBUG_SITE_MASS_GUIDE);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (PDV_LD(Sq, mid, n_v + 1, PDV_DEBUG_SITE_MASS_NODE) <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float term) {
  const float y = term - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Launch position on the beam disk (event 0 of the packet's stream). Only the
// detection test needs it, so it is drawn when a packet reaches the probe.
__device__ __forceinline__ void launch_position(unsigned long long pk, unsigned sid, uint2 key,
                                                float r_beam, float& x0, float& y0) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)pk, (unsigned)(pk >> 32), 0u, sid), key);
  const float rad = r_beam * sqrtf(u23f(r.x));
  float sp, cp;
  sincospif(2.0f * u23f(r.y), &sp, &cp);
  x0 = rad * cp;
  y0 = rad * sp;
}

#ifdef PDV_DEBUG
// Debug build: one vertex of a traced packet's path (pdv_debug_set_trace).
__device__ __noinline__ static void trace_put(const SetDesc& sd, unsigned long long off,
                                              unsigned& nv, double x, double y, double z, double v,
                                              double ux, double uy, double uz, int kind,
                                              unsigned ev) {
  if (sd.trace == nullptr || off >= (unsigned long long)sd.n_trace) return;
  if (nv < (unsigned)sd.max_vtx) {
    pdv_trace_vertex e;
    e.x = x; e.y = y; e.z = z; e.v = v;
    e.ux = ux; e.uy = uy; e.uz = uz;
    e.kind = kind;
    e.event = ev;
    sd.trace[off * (unsigned long long)sd.max_vtx + nv] = e;
  }
  ++nv;
}
#endif

// Stage one set's tables (and a cleared private histogram) in shared memory.
template <int HMODE>
__device__ __forceinline__ SmemTables stage_set(const SetDesc& sd, unsigned char* smem) {
  size_t off[12];
  smem_layout(sd.n_v, sd.n_g, sd.n_p, sd.n_snap, sd.n_bins, HMODE, sd.phase_uniform, sd.ap_all,
              sd.expo, sd.angle_table, off);
  SmemTables tb;
  tb.Sq = reinterpret_cast<const unsigned long long*>(smem + off[0]);
  tb.w = reinterpret_cast<const float*>(smem + off[1]);
  tb.G = reinterpret_cast<const unsigned short*>(smem + off[2]);
  tb.node = reinterpret_cast<const uint2*>(smem + off[3]);
  tb.thpi = reinterpret_cast<const float*>(smem + off[4]);
  tb.dthpi = reinterpret_cast<const float*>(smem + off[5]);
  tb.Gp = reinterpret_cast<const unsigned short*>(smem + off[6]);
  tb.ts = reinterpret_cast<const float*>(smem + off[7]);
  tb.perm = reinterpret_cast<const unsigned short*>(smem + off[8]);
  tb.hist = HMODE == 2 ? reinterpret_cast<unsigned long long*>(smem + off[9]) : sd.hist;
  tb.ang = reinterpret_cast<const float2*>(smem + off[10]);
  tb.turn = reinterpret_cast<const float2*>(smem + off[11]);
  {
    if (!sd.expo) {
      unsigned long long* Sq = reinterpret_cast<unsigned long long*>(smem + off[0]);
      for (int i = threadIdx.x; i <= sd.n_v; i += blockDim.x) Sq[i] = sd.Sq[i];
      float* w = reinterpret_cast<float*>(smem + off[1]);
      for (int i = threadIdx.x; i < sd.n_v; i += blockDim.x) w[i] = sd.w[i];
      unsigned short* G = reinterpret_cast<unsigned short*>(smem + off[2]);
      for (int i = threadIdx.x; i <= sd.n_g; i += blockDim.x) G[i] = sd.G[i];
    }
    uint2* node = reinterpret_cast<uint2*>(smem + off[3]);
    float* thpi = reinterpret_cast<float*>(smem + off[4]);
    float* dthpi = reinterpret_cast<float*>(smem + off[5]);
    float2* ang = reinterpret_cast<float2*>(smem + off[10]);
    float2* turn = reinterpret_cast<float2*>(smem + off[11]);
    for (int j = threadIdx.x; j < kTurn; j += blockDim.x) {
      float sj, cj;
      sincospif((float)j * (2.0f / (float)kTurn), &sj, &cj);   // exact argument 2 j / kTurn
      turn[j] = make_float2(cj, sj);
    }
    for (int i = threadIdx.x; i < sd.n_p; i += blockDim.x) {
      node[i] = sd.node[i];
      ang[i] = sd.cs[i];
      if (!sd.phase_uniform && !sd.angle_table) {
        thpi[i] = sd.thpi[i];
        dthpi[i] = sd.dthpi[i];
      }
    }
    unsigned short* Gp = reinterpret_cast<unsigned short*>(smem + off[6]);
    for (int i = threadIdx.x; i <= (1 << kGuidePhaseLog); i += blockDim.x) Gp[i] = sd.Gp[i];
    float* ts = reinterpret_cast<float*>(smem + off[7]);
    unsigned short* perm = reinterpret_cast<unsigned short*>(smem + off[8]);
    for (int i = threadIdx.x; i < sd.n_snap; i += blockDim.x) {
      ts[i] = (float)sd.t_snap[sd.n_snap + i];
      perm[i] = (unsigned short)sd.t_snap[2 * sd.n_snap + i];
    }
    if (HMODE == 2) {
      unsigned long long* h = reinterpret_cast<unsigned long long*>(smem + off[9]);
      const int nh = tally_rows(sd.n_snap, sd.ap_all) * hist_row(sd.n_bins);
      for (int i = threadIdx.x; i < nh; i += blockDim.x) h[i] = 0ull;
    }
  }
  __syncthreads();
  return tb;
}

// The walks of one set by this block's warps (Section II.B steps (1)-(7)),
// with the per-set sums added to the block's counters s_cnt. FAST: every set
// of the launch has the configuration transport_fast_set names, so the walk
// takes its branches at compile time instead of testing the set's switches
// every flight.
template <bool DUMP, int HMODE, bool IMPL, bool FAST>
__device__ __forceinline__ void walk_set(const SetDesc& sd, const SmemTables& tb,
                                         unsigned long long* __restrict__ ctr, unsigned chunk,
                                         unsigned long long* s_cnt) {
  const int lane = threadIdx.x & 31;
  // ---- per-set constants in registers
  const uint2 key = make_uint2((unsigned)sd.seed, (unsigned)(sd.seed >> 32));
  const unsigned sid = sd.stream_id;
  const unsigned long long base_pk = sd.packet_begin;
  const unsigned n_pk = (unsigned)sd.n_packets;    // at most 4e9 packets per set
  const float inv_tau = sd.inv_tau_f;
  const int n_bins = sd.n_bins, row = hist_row(sd.n_bins), n_snap = sd.n_snap;
  // sizes of the staged tables and of the tally (the debug build checks against them)
  const int n_p = sd.n_p;
  const long long n_tally = (long long)tally_rows(n_snap, sd.ap_all) * row;
#ifdef PDV_DEBUG
  unsigned n_vtx = 0;                               // vertices of this lane's traced packet
#else
  (void)n_p;
  (void)n_tally;
#endif

  // ---- warp loop
  // The warp owns a chunk [pool_next, pool_end) of packet offsets and has the
  // next chunk's claim already in flight (lane 0's `pre`), so the global
  // atomic's latency is hidden behind a chunk's worth of events.
  unsigned pool_next = 0, pool_end = 0;
  unsigned long long pre = 0;
  if (lane == 0) pre = atomicAdd(ctr, (unsigned long long)chunk);
  bool exhausted = false, alive = false;
  unsigned long long pk = 0, W = 0;
  long long Sq = 0;
  // kev: index of the flight's Philox block (1 for the first flight); the
  // packet has made kev - 1 events when a flight that is an event starts
  unsigned kev = 0, nsca = 0, nsurf = 0;
  unsigned long long dmask = 0;
  float vcur = 0.f, ux = 0.f, uy = 0.f, uz = -1.f, iuz = -1.f;
  float Xx = 0.f, Xy = 0.f, vapp = 0.f, vcomp = 0.f;
  // w_launch: packets this warp launched (the same in every lane)
  unsigned w_launch = 0, st_events = 0, st_scat = 0, st_surf = 0, st_esc = 0;
  unsigned long long st_wesc = 0, st_wabs = 0, st_wsurf = 0;   // escaped / absorbed weight

  const unsigned lt_mask = lanemask_lt();
  for (;;) {
    // refill dead lanes from the warp's chunk of packets, in one pass: when
    // the chunk runs out, the lanes it could not serve wait one flight
    const unsigned need = __ballot_sync(kFull, !alive);
    if (need) {
      unsigned avail = pool_end - pool_next;
      if (avail == 0 && !exhausted) {
        const unsigned long long b = __shfl_sync(kFull, pre, 0);
        if (b >= (unsigned long long)n_pk) {
          exhausted = true;
        } else {
          if (lane == 0) pre = atomicAdd(ctr, (unsigned long long)chunk);
          pool_next = (unsigned)b;
          pool_end = n_pk - pool_next > chunk ? pool_next + chunk : n_pk;
          avail = pool_end - pool_next;
        }
      }
      const unsigned cnt = __popc(need);
      const unsigned take = avail < cnt ? avail : cnt;
      const unsigned rank = __popc(need & lt_mask);
      if (!alive && rank < take) {
        // Step (1): a new packet at the top of the cloud moving along -z
        pk = base_pk + (pool_next + rank);
        ux = 0.f; uy = 0.f; uz = -1.f; iuz = -1.f;
        if (!FAST && sd.launch_horizontal) {      // test hook: the horizontal-flight rule
          ux = 1.f; uz = 0.f; iuz = 0.f;
        }
        Sq = (long long)kOneQ;
        vcur = sd.v_top_f;
        Xx = 0.f; Xy = 0.f; vapp = 0.f; vcomp = 0.f;
        W = 1ull << 32;
        kev = 1;
        if (DUMP) { nsca = 0; nsurf = 0; dmask = 0; }
        alive = true;
#ifdef PDV_DEBUG
        if (sd.debug_check && pk == base_pk)     // PDV_TEST_DEBUG_CHECK: once per set
          (void)PDV_IN(n_tally, n_tally, PDV_DEBUG_SITE_SELFTEST);
        if (DUMP && sd.trace) {
          float x0, y0;
          launch_position(pk, sid, key, sd.r_beam_f, x0, y0);
          n_vtx = 0;
          trace_put(sd, pk - base_pk, n_vtx, x0, y0, sd.z_probe_f, 0.0, ux, uy, uz, 0, 0u);
        }
#endif
      }
      pool_next += take;
      w_launch += take;
    }
    if (!__any_sync(kFull, alive)) break;

    // ---- one flight and what ends it. Every lane runs the same straight
    // line; the outcome's predicates select what each lane commits, and a
    // lane without a packet (at the end of a set) commits nothing.
    const uint4 r = philox4x32_10_rk(make_uint4((unsigned)pk, (unsigned)(pk >> 32), kev, sid), sd.rk);
    ++kev;
    const float tau = -logf(u23f(r.x));                // Step (3): Beer–Lambert
    const float dS = tau * uz * inv_tau;
    const bool horiz = fabsf(uz) < 1e-9f;
    // dS 2^62 truncated towards zero, exactly (a power-of-two scaling, then a
    // 64-bit conversion); the largest binary32 magnitude below 1 keeps it in
    // range, and a flight of |dS| >= 1 leaves the cloud whatever its end
    long long Sn =
        Sq + __float2ll_rz(fminf(fmaxf(dS, -0.99999994f), 0.99999994f) * 4.611686018427388e18f);
    // 0 interaction, 1 escape through the top, 2 free surface; a horizontal
    // flight is an interaction where it started (set in the lateral move below)
    int what = (dS >= 1.0f || Sn >= (long long)kOneQ) ? 1 : ((dS <= -1.0f || Sn <= 0) ? 2 : 0);
    // velocity coordinate z/t where the flight ends
    float vn = vcur;
    if (FAST || sd.expo) {
      // Eq. 20 inverted in closed form: v = v_fs (1 - ln((1 - S) + S eps) / beta); 1 - S is
      // exact in the fixed-point state, so the top of the cloud keeps its relative precision
      // (32-bit conversions: the 64-bit ones run on the FP64 pipe)
      const unsigned long long sn = (unsigned long long)Sn, oms = kOneQ - sn;
      const float om = fmaf(__uint2float_rn((unsigned)(oms >> 32)), kTwoM30f,
                            __uint2float_rn((unsigned)oms) * kTwoM62f);
      const float q = fmaf(__uint2float_rn((unsigned)(sn >> 32)), sd.eps30_f, om);
      vn = fmaf(-sd.lg_c_f, __log2f(q), sd.v_fs_f);
    } else if (what == 0) {
      const int j = search_mass(tb.Sq, tb.G, sd.g_shift, sd.n_g, sd.n_v, (unsigned long long)Sn);
      const float fd =
          u64_to_f((unsigned long long)Sn - PDV_LD(tb.Sq, j, sd.n_v + 1, PDV_DEBUG_SITE_MASS_NODE));
      vn = fmaf(fd, PDV_LD(tb.w, j, sd.n_v, PDV_DEBUG_SITE_MASS_NODE),
                fmaf((float)j, sd.dv_f, sd.v_bot_f));
    }
    vn = what == 1 ? sd.v_top_f : (what == 2 ? sd.v_fs_f : vn);
    // lateral displacement in velocity units (x = x0 + t X)
    if (!horiz) {
      const float d = vn - vcur;
      // (x, y) pairs as packed FP32x2 products (each half rounds as fmaf / fmul)
      const float2 X = __ffma2_rn(__fmul2_rn(make_float2(ux, uy), make_float2(iuz, iuz)),
                                  make_float2(d, d), make_float2(Xx, Xy));
      Xx = X.x;
      Xy = X.y;
    } else {
      // horizontal packet: lateral path tau / mu(z), in velocity units tau / tau_tot dv/dS
      float dvds;
      if (FAST || sd.expo) {
        const unsigned long long sq = (unsigned long long)Sq, oms = kOneQ - sq;
        const float om = fmaf(__uint2float_rn((unsigned)(oms >> 32)), kTwoM30f,
                              __uint2float_rn((unsigned)oms) * kTwoM62f);
        dvds = sd.dvds_c_f / fmaf(__uint2float_rn((unsigned)(sq >> 32)), sd.eps30_f, om);
      } else {
        const int j = search_mass(tb.Sq, tb.G, sd.g_shift, sd.n_g, sd.n_v, (unsigned long long)Sq);
        dvds = PDV_LD(tb.w, j, sd.n_v, PDV_DEBUG_SITE_MASS_NODE) * 4.611686018427388e18f;
      }
      const float len = tau * inv_tau * dvds;
      Xx = fmaf(ux, len, Xx);
      Xy = fmaf(uy, len, Xy);
      // the interaction happens at the starting depth, velocity unchanged
      Sn = Sq;
      vn = vcur;
      what = 0;
    }

    // ---- Step (6): out through the top, vacuum flight to the probe plane
    const bool esc = alive && what == 1;
    const bool cone = esc && (sd.cone_all || uz >= sd.cos_alpha_f);
    if (cone) {
      // v_app is summed doubled (below); the exact scalings undo it
      const float fb = floorf((vapp - vcomp - 2.0f * sd.v_lo_f) * (0.5f * sd.inv_dbin_f));
      const int idx = fb < 0.0f ? 0 : (fb >= (float)n_bins ? n_bins + 1 : (int)fb + 1);
      if (sd.ap_all) {
        // Eq. 19 at every snapshot time alike (unlimited aperture): one
        // tally in row 0, which the normalisation reads for each time
        if (PDV_IN(idx, n_tally, PDV_DEBUG_SITE_HISTOGRAM)) atomicAdd(&tb.hist[idx], W);
        if (PDV_IN(n_bins + 2, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
          atomicAdd(&tb.hist[n_bins + 2], 1ull);
        if (DUMP) dmask = n_snap >= 64 ? ~0ull : ((1ull << n_snap) - 1ull);
      } else {
        float x0, y0;
        launch_position(pk, sid, key, sd.r_beam_f, x0, y0);
        const float tx = ux * iuz, ty = uy * iuz;
        const float ax = fmaf(tx, sd.z_probe_f, x0), ay = fmaf(ty, sd.z_probe_f, y0);
        const float bx = fmaf(-tx, sd.v_top_f, Xx), by = fmaf(-ty, sd.v_top_f, Xy);
        // |a + t b|^2 <= R^2 holds on one interval of t: visit the ascending
        // snapshot times inside it, plus one on each side, each re-tested
        // exactly as below (the interval only narrows the search)
        int s0 = 0, s1 = n_snap;
        const float A = fmaf(bx, bx, by * by);
        const float B = 2.0f * fmaf(ax, bx, ay * by);
        const float Cc = fmaf(ax, ax, fmaf(ay, ay, -sd.r_ap2_f));
        const float disc = fmaf(B, B, -4.0f * A * Cc);
        if (A > 0.0f) {
          if (disc < 0.0f) {
            s1 = 0;
          } else {
            const float q = sqrtf(disc), ia = 0.5f / A;
            const float t1 = (-B - q) * ia, t2 = (-B + q) * ia;
            int lo = 0, hi = n_snap;                   // first time >= t1
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (PDV_LD(tb.ts, mid, n_snap, PDV_DEBUG_SITE_SNAPSHOT) < t1) lo = mid + 1; else hi = mid;
            }
            s0 = lo > 0 ? lo - 1 : 0;
            hi = n_snap;                               // first time > t2
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (PDV_LD(tb.ts, mid, n_snap, PDV_DEBUG_SITE_SNAPSHOT) <= t2) lo = mid + 1; else hi = mid;
            }
            s1 = lo < n_snap ? lo + 1 : n_snap;
          }
        }
        for (int s = s0; s < s1; ++s) {
          const float t = PDV_LD(tb.ts, s, n_snap, PDV_DEBUG_SITE_SNAPSHOT);
          const float dx = fmaf(t, bx, ax), dy = fmaf(t, by, ay);
          if (fmaf(dx, dx, dy * dy) <= sd.r_ap2_f) {
            // Eq. 19: tally the out-photon at its frequency shift
            const int sr = PDV_LD(tb.perm, s, n_snap, PDV_DEBUG_SITE_SNAPSHOT);
            if (PDV_IN((long long)sr * row + idx, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
              atomicAdd(&tb.hist[(size_t)sr * row + idx], W);
            if (PDV_IN((long long)sr * row + n_bins + 2, n_tally, PDV_DEBUG_SITE_HISTOGRAM))
              atomicAdd(&tb.hist[(size_t)sr * row + n_bins + 2], 1ull);
            if (DUMP && sr < 64) dmask |= 1ull << sr;
          }
        }
      }
    }
    st_esc += esc ? 1u : 0u;
    st_wesc += esc ? W : 0ull;

    // ---- an event: interaction (what 0) or the free surface (what 2)
    const bool ev = alive && what != 1;
    const bool surf = ev && what == 2;
    if (ev) {
      Sq = what == 2 ? 0ll : Sn;
      vcur = vn;
      ++st_events;
    }
    // Step (6): free surface z = v_fs t, reflectivity in 2^32 fixed point:
    // round(W R_q / 2^32). W <= 2^32, and R_q < 2^32 unless R = 1, so the
    // product is one 32 x 32 -> 64-bit multiply-add; W = 2^32 gives R_q.
    // as ((W - 1) R_q + R_q + 2^31) >> 32: one multiply-add for every W in
    // [1, 2^32] (W - 1 fits 32 bits), W = 2^32 included
    const unsigned long long Wr =
        (!FAST && sd.R_q >= (1ull << 32))
            ? W
            : ((unsigned long long)((unsigned)W - 1u) * (unsigned)sd.R_q + (sd.R_q + (1ull << 31))) >> 32;
    st_surf += surf ? 1u : 0u;
    if (DUMP) nsurf += surf ? 1u : 0u;
    const unsigned long long Ws = surf ? Wr : W;   // the weight after the flight's end
    st_wsurf += W - Ws;
    W = Ws;
    // Eq. 11: analog absorption (the gate is omega_q). Implicit capture (gate
    // 0): the particle absorbs 1 - omega of the weight and the packet
    // scatters; a light packet plays the roulette on r1. Launches without
    // implicit sets compile this out.
    const bool absorb = ev && !surf && (r.y >> 8) >= (IMPL ? sd.absorb_gate : sd.omega_q);
    unsigned fate = esc ? 1u : 0u;
    if (!IMPL) {
      st_wabs += absorb ? W : 0ull;
      fate = absorb ? 2u : fate;
    } else if (absorb) {
      if (!sd.implicit) {
        st_wabs += W;
        fate = 2;
      } else {
        const unsigned long long Wn = (W * sd.omega_q + (1ull << 23)) >> 24;
        st_wabs += W - Wn;
        W = Wn;
        if (Wn < PDV_ROULETTE_W) {
          if (Wn != 0 && (r.y >> 8) < PDV_ROULETTE_Q) {
            atomicAdd(&s_cnt[C_W_RR_GAINED], (PDV_ROULETTE_M - 1) * Wn);
            W = Wn * PDV_ROULETTE_M;
          } else {
            atomicAdd(&s_cnt[C_W_RR_DROPPED], Wn);
            fate = 5;
          }
        }
      }
    }

    // ---- new direction. Particle scattering (Eq. 13-17): polar angle from
    // the phase CDF, azimuth uniform (Eq. 15). Free surface (diffuse): polar
    // angle uniform in [0, pi/2) from +z, azimuth uniform. Both are a
    // (polar, azimuth) pair in units of pi followed by the same rotation.
    const bool scat = ev && fate == 0;
    const bool part = scat && !surf;
    // polar angle as a table node plus a remainder d: a particle's from its
    // phase-CDF bin (theta_i + frac (theta_{i+1} - theta_i)), the wall's
    // theta' = (pi/2) u from the turn table at a quarter of a turn. Phase
    // tables with a node spacing above 3.1e-3 (where d^4/24 would matter)
    // take sin/cos of the angle in half turns instead.
    float st, ct, sp, cp;
    {
      const unsigned m2 = r.z >> 8;
      const unsigned c = m2 >> (24 - kGuidePhaseLog);
      constexpr int n_gp = (1 << kGuidePhaseLog) + 1;
      int lo = PDV_LD(tb.Gp, c, n_gp, PDV_DEBUG_SITE_PHASE_GUIDE);
      int hi = part ? (int)PDV_LD(tb.Gp, c + 1, n_gp, PDV_DEBUG_SITE_PHASE_GUIDE) : lo;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (PDV_LD(tb.node, mid, n_p, PDV_DEBUG_SITE_PHASE_NODE).x <= m2) lo = mid; else hi = mid - 1;
      }
      const uint2 nd = PDV_LD(tb.node, lo, n_p, PDV_DEBUG_SITE_PHASE_NODE);
      const float fm = (float)(m2 - nd.x) + 0.5f;
      if (FAST || sd.angle_table) {
        // theta = theta_i + d with d = (m - Cq_i + 1/2) times the bin's slope
        const float dp = fm * __uint_as_float(nd.y);
        // theta' = 2 pi f with f = u / 4 = ((r1 >> 9) + 1/2) 2^-25: the nearest
        // table step j and the remainder, both exact in integers
        const int m1 = (int)(r.y >> 9);
        const int js = (m1 + (1 << 14)) >> 15;
        const float ds = (float)(2 * (m1 - (js << 15)) + 1) * kPi2m25f;
        // one load: the node's (cos, sin), or the wall's turn step
        cos_sin_add(PDV_LD(tb.ang, surf ? n_p + js : lo, n_p + kTurn, PDV_DEBUG_SITE_PHASE_NODE),
                    surf ? ds : dp, &ct, &st);
      } else {
        // theta_i / pi = i / (n_p - 1) on a uniform grid; linear inside the CDF bin
        const float tp =
            sd.phase_uniform
                ? ((float)lo +
                   fm * rcp_approx(
                            (float)(PDV_LD(tb.node, lo + 1, n_p, PDV_DEBUG_SITE_PHASE_NODE).x - nd.x))) *
                      sd.inv_nm1
                : fmaf(fm, PDV_LD(tb.dthpi, lo, n_p, PDV_DEBUG_SITE_PHASE_NODE),
                       PDV_LD(tb.thpi, lo, n_p, PDV_DEBUG_SITE_PHASE_NODE));
        sincospi_half_turns(surf ? 0.5f * u23f(r.y) : tp, &st, &ct);
      }
    }
    {
      // azimuth, Eq. 15: phi = 2 pi u with u = ((r >> 9) + 1/2) 2^-23
      // the nearest of the kTurn steps, jp = ((r >> 9) + 2^12) >> 13 modulo kTurn, and the
      // remainder (r >> 9) - jp 2^13 in [-2^12, 2^12): bits 9-21 of r, sign-extended
      const unsigned rw = surf ? r.z : r.w;
      const unsigned jp = (rw + (1u << 21)) >> 22;
      const int rem = (int)(rw << 10) >> 19;
      const float dphi = (float)(2 * rem + 1) * kPi2m23f;
      cos_sin_add(tb.turn[jp], dphi, &cp, &sp);
    }
    if (!FAST && sd.surface_mode == PDV_SURFACE_LAMBERT) {
      const float a = u23f(r.y);
      ct = surf ? sqrtf(a) : ct;
      st = surf ? sqrtf(1.0f - a) : st;
    }
    // Eq. 16 in its standard form, with the horizontal norm from (u_x, u_y);
    // Eq. 17 (and the wall's frame) when the direction is vertical (its
    // horizontal part below 1e-15): cos(theta) along the sign of u_z
    const float h2 = fmaf(ux, ux, uy * uy);
    const bool vert = surf || h2 < 1e-30f;
    const float rs = rsqrtf(h2);
    const float sh = h2 * rs;
    const float ah = st * rs;
    // the horizontal part as one complex product, (n_x + i n_y) = (u_x + i u_y)
    // (ct + ah u_z cp + i ah sp): Eq. 16's terms grouped, three products fewer
    const float ga = fmaf(ah * uz, cp, ct), gb = ah * sp;
    float nx = fmaf(ux, ga, -uy * gb);
    float ny = fmaf(uy, ga, ux * gb);
    float nz = fmaf(-st * cp, sh, uz * ct);
    nx = vert ? st * cp : nx;
    ny = vert ? st * sp : ny;
    nz = vert ? ((surf || uz >= 0.0f) ? ct : -ct) : nz;
    const bool spec = !FAST && surf && sd.surface_mode == PDV_SURFACE_SPECULAR;
    const float inv_n = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    const float2 nn = __fmul2_rn(make_float2(nx, ny), make_float2(inv_n, inv_n));
    nx = spec ? ux : nn.x;
    ny = spec ? uy : nn.y;
    nz = spec ? -uz : nz * inv_n;
    if (scat) {
      // Eq. 4 / Eq. 18: the moving scatterer (or wall) shifts the frequency
      // (a rounded product: no FMA contraction into the compensated sum,
      // so every instantiation of this kernel computes the same bits)
      kahan_add(vapp, vcomp, __fmul_rn(nz - uz, vn));   // 2 v_app: the half applied at the end
      ux = nx; uy = ny; uz = nz;
      iuz = rcp_approx(nz);
    }
    st_scat += part ? 1u : 0u;
    if (DUMP) nsca += part ? 1u : 0u;
    fate = (scat && W == 0) ? 3u : fate;     // the surface absorbed all of the weight
    // the event limit: kev (already advanced) exceeds max_events once the
    // packet has made max_events events
    if (fate == 0 && ev && kev > sd.max_events) {
      atomicAdd(&s_cnt[C_W_TRUNCATED], W);
      atomicAdd(&s_cnt[C_TRUNCATED], 1ull);
      fate = 4;
    }
#ifdef PDV_DEBUG
    if (DUMP && alive && sd.trace && pk - base_pk < (unsigned long long)sd.n_trace) {
      // the vertex that ended this flight, at the first snapshot time
      float x0, y0;
      launch_position(pk, sid, key, sd.r_beam_f, x0, y0);
      const float t = (float)sd.t_trace;
      if (esc) {
        const float zt = sd.v_top_f * t;
        trace_put(sd, pk - base_pk, n_vtx, fmaf(ux * iuz, sd.z_probe_f - zt, fmaf(t, Xx, x0)),
                  fmaf(uy * iuz, sd.z_probe_f - zt, fmaf(t, Xy, y0)), sd.z_probe_f, 0.0, ux, uy, uz, 3,
                  kev - 1);
      } else if (ev) {
        trace_put(sd, pk - base_pk, n_vtx, fmaf(t, Xx, x0), fmaf(t, Xy, y0), vn * t, vn, ux, uy, uz,
                  surf ? 2 : (scat ? 1 : 4), kev - 1);
      }
    }
#endif
    if (fate) {
      if (DUMP && sd.packets) {
        pdv_packet_record rec;
        rec.n_events = kev - 1u - (fate == 1u ? 1u : 0u);
        rec.n_scatters = nsca;
        rec.n_surface = nsurf;
        rec.fate = fate;
        rec.weight = W;
        rec.v_app = 0.5 * ((double)vapp - (double)vcomp);
        rec.detect_mask = dmask;
        if (PDV_IN(pk - base_pk, sd.n_packets, PDV_DEBUG_SITE_PACKET)) sd.packets[pk - base_pk] = rec;
      }
      alive = false;
    }
  }

  // ---- flush this set's tallies
  {
    unsigned b = st_events, c = st_scat, d = st_surf, e = st_esc;
    unsigned long long we = st_wesc, wa = st_wabs, ws = st_wsurf;
    for (int o = 16; o; o >>= 1) {
      b += __shfl_xor_sync(kFull, b, o);
      c += __shfl_xor_sync(kFull, c, o);
      d += __shfl_xor_sync(kFull, d, o);
      e += __shfl_xor_sync(kFull, e, o);
      we += __shfl_xor_sync(kFull, we, o);
      wa += __shfl_xor_sync(kFull, wa, o);
      ws += __shfl_xor_sync(kFull, ws, o);
    }
    if (lane == 0) {
      atomicAdd(&s_cnt[C_LAUNCHED], (unsigned long long)w_launch);
      atomicAdd(&s_cnt[C_EVENTS], (unsigned long long)b);
      atomicAdd(&s_cnt[C_SCATTERS], (unsigned long long)c);
      atomicAdd(&s_cnt[C_SURFACE_HITS], (unsigned long long)d);
      atomicAdd(&s_cnt[C_ESCAPES], (unsigned long long)e);
      atomicAdd(&s_cnt[C_W_ESCAPED], we);
      atomicAdd(&s_cnt[C_W_ABS_PARTICLE], wa);
      atomicAdd(&s_cnt[C_W_ABS_SURFACE], ws);
    }
  }
}

// The block's counters and private histogram into the set's global tallies.
template <int HMODE>
__device__ __forceinline__ void flush_set(const SetDesc& sd, const SmemTables& tb,
                                          const unsigned long long* s_cnt) {
  if (threadIdx.x < C_NCOUNT && s_cnt[threadIdx.x])
    atomicAdd(&sd.cnt[threadIdx.x], s_cnt[threadIdx.x]);
  if (HMODE == 2) {
    const int nh = tally_rows(sd.n_snap, sd.ap_all) * hist_row(sd.n_bins);
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
      const unsigned long long v = tb.hist[i];
      if (v && PDV_IN(i, (long long)sd.n_snap * hist_row(sd.n_bins), PDV_DEBUG_SITE_HISTOGRAM))
        atomicAdd(&sd.hist[i], v);
    }
  }
}

// Persistent launch over a list of sets (batches and serving): blocks walk the
// list from their own offset and stay on a set until its packets are claimed.
template <bool DUMP, int HMODE, bool IMPL, bool FAST>
__global__ void __launch_bounds__(256, 4) k_transport_f32(const SetDesc* __restrict__ sets,
                                                          int n_sets,
                                                          unsigned long long* __restrict__ set_ctr,
                                                          unsigned chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SetDesc sd;
  __shared__ unsigned long long s_cnt[C_NCOUNT];
  __shared__ int s_go;
  const int start = (int)(((long long)blockIdx.x * n_sets) / gridDim.x);
  for (int step = 0; step < n_sets; ++step) {
    const int si = (start + step) % n_sets;
    if (threadIdx.x == 0) {
      const unsigned long long c = *((volatile unsigned long long*)&set_ctr[si]);
      s_go = c < sets[si].n_packets;
    }
    __syncthreads();
    const int go = s_go;
    __syncthreads();
    if (!go) continue;
    {
      const int* src = reinterpret_cast<const int*>(&sets[si]);
      int* dst = reinterpret_cast<int*>(&sd);
      for (int i = threadIdx.x; i < (int)(sizeof(SetDesc) / sizeof(int)); i += blockDim.x)
        dst[i] = src[i];
      if (threadIdx.x < C_NCOUNT) s_cnt[threadIdx.x] = 0ull;
    }
    __syncthreads();
    const SmemTables tb = stage_set<HMODE>(sd, smem);
    __syncthreads();
    walk_set<DUMP, HMODE, IMPL, FAST>(sd, tb, &set_ctr[si], chunk, s_cnt);
    __syncthreads();
    flush_set<HMODE>(sd, tb, s_cnt);
    __syncthreads();
  }
}

// Persistent launch of one set whose descriptor is a kernel parameter: the
// walk reads its constants (and Philox's round keys) as constant-bank
// operands instead of shared-memory loads and registers.
template <bool DUMP, int HMODE, bool IMPL, bool FAST>
__global__ void __launch_bounds__(256, 4) k_transport_f32_one(const __grid_constant__ SetDesc sd,
                                                              unsigned long long* __restrict__ ctr,
                                                              unsigned chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_cnt[C_NCOUNT];
  if (threadIdx.x < C_NCOUNT) s_cnt[threadIdx.x] = 0ull;
  const SmemTables tb = stage_set<HMODE>(sd, smem);
  __syncthreads();
  walk_set<DUMP, HMODE, IMPL, FAST>(sd, tb, ctr, chunk, s_cnt);
  __syncthreads();
  flush_set<HMODE>(sd, tb, s_cnt);
}

// The configuration the FAST builds take at compile time: the exponential law
// (closed-form velocity), sin/cos from the node table, the diffuse wall with
// the polar angle uniform in [0, pi/2) and R < 1, no horizontal launch.
bool transport_fast_set(const SetDesc& d) {
  return d.expo && d.angle_table && !d.launch_horizontal &&
         d.surface_mode == PDV_SURFACE_UNIFORM_THETA && d.R_q < (1ull << 32);
}

template <bool IMPL, bool FAST>
static const void* f32_kernel_hm(int hist_mode, bool one) {
  if (one)
    return hist_mode == 2 ? (const void*)k_transport_f32_one<false, 2, IMPL, FAST>
                          : (const void*)k_transport_f32_one<false, 1, IMPL, FAST>;
  return hist_mode == 2 ? (const void*)k_transport_f32<false, 2, IMPL, FAST>
                        : (const void*)k_transport_f32<false, 1, IMPL, FAST>;
}

template <bool IMPL>
static const void* f32_kernel_impl(int hist_mode, bool dump, bool one, bool fast) {
  if (dump) {                      // packet dumps: the generic build
    if (one)
      return hist_mode == 2 ? (const void*)k_transport_f32_one<true, 2, IMPL, false>
                            : (const void*)k_transport_f32_one<true, 1, IMPL, false>;
    return hist_mode == 2 ? (const void*)k_transport_f32<true, 2, IMPL, false>
                          : (const void*)k_transport_f32<true, 1, IMPL, false>;
  }
  return fast ? f32_kernel_hm<IMPL, true>(hist_mode, one) : f32_kernel_hm<IMPL, false>(hist_mode, one);
}

static const void* f32_kernel(int hist_mode, bool dump, bool impl, bool one, bool fast) {
  return impl ? f32_kernel_impl<true>(hist_mode, dump, one, fast)
              : f32_kernel_impl<false>(hist_mode, dump, one, fast);
}

__global__ void k_normalise(const SetDesc* __restrict__ sets, double* const* spec,
                            pdv_counters* const* cnt_out, unsigned long long* const* raw,
                            const unsigned* flags);

cudaError_t transport_preload() {
  cudaFuncAttributes a;
  for (int one = 0; one < 2; ++one)
    for (int impl = 0; impl < 2; ++impl)
      for (int dump = 0; dump < 2; ++dump)
        for (int hm = 1; hm <= 2; ++hm)
          for (int fast = 0; fast < 2; ++fast) {
            const cudaError_t e = cudaFuncGetAttributes(
                &a, f32_kernel(hm, dump != 0, impl != 0, one != 0, fast != 0));
            if (e != cudaSuccess) return e;
          }
  return cudaFuncGetAttributes(&a, (const void*)k_normalise);
}

int transport_f32_max_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v - (int)(sizeof(SetDesc) + sizeof(unsigned long long) * C_NCOUNT + 64);
}

cudaError_t transport_f32_occupancy(int block, size_t smem, int hist_mode, bool dump, bool impl,
                                    bool one, bool fast, int* blocks) {
  const void* k = f32_kernel(hist_mode, dump, impl, one, fast);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, block, smem);
}

void launch_transport_f32(const SetDesc* d_sets, int n_sets, unsigned long long* d_set_ctr,
                          int grid, int block, size_t smem, int hist_mode, bool dump, bool impl,
                          bool fast, unsigned chunk, cudaStream_t st) {
  const void* k = f32_kernel(hist_mode, dump, impl, false, fast);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (chunk == 0) chunk = kChunkDefault;
  void* args[] = {(void*)&d_sets, (void*)&n_sets, (void*)&d_set_ctr, (void*)&chunk};
  cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

void launch_transport_f32_one(const SetDesc& sd, unsigned long long* d_ctr, int grid, int block,
                              size_t smem, int hist_mode, bool dump, bool impl, bool fast,
                              unsigned chunk, cudaStream_t st) {
  const void* k = f32_kernel(hist_mode, dump, impl, true, fast);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (chunk == 0) chunk = kChunkDefault;
  SetDesc arg = sd;
  void* args[] = {(void*)&arg, (void*)&d_ctr, (void*)&chunk};
  cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

// ------------------------------------------------------------------ FP64
__device__ int search_mass_d(const double* Sd, int n_v, double s) {
  int lo = 0, hi = n_v - 1;                      // largest j <= n_v-1 with Sd_j <= s
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (PDV_LD(Sd, mid, n_v + 1, PDV_DEBUG_SITE_MASS_NODE) <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_transport_f64(const SetDesc* __restrict__ setp) {
  __shared__ unsigned long long s_cnt[C_NCOUNT];
  if (threadIdx.x < C_NCOUNT) s_cnt[threadIdx.x] = 0ull;
  __syncthreads();
  const SetDesc& sd = *setp;
  const double pi = 3.14159265358979323846;
  const uint2 key = make_uint2((unsigned)sd.seed, (unsigned)(sd.seed >> 32));
  const int n_bins = sd.n_bins, row = hist_row(n_bins);
  unsigned long long st_launch = 0, st_events = 0, st_scat = 0, st_surf = 0;
  for (unsigned long long ip = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       ip < sd.n_packets; ip += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long pk = sd.packet_begin + ip;
    uint4 r = philox4x32_10(make_uint4((unsigned)pk, (unsigned)(pk >> 32), 0u, sd.stream_id), key);
    const double rad = sd.r_beam * sqrt(u23d(r.x));
    const double psi = 2.0 * pi * u23d(r.y);
    const double x0 = rad * cos(psi), y0 = rad * sin(psi);
    double ux = 0.0, uy = 0.0, uz = -1.0;
    if (sd.launch_horizontal) {          // test hook: the horizontal-flight rule
      ux = 1.0;
      uz = 0.0;
    }
    double S = 1.0, vcur = sd.v_top, Xx = 0.0, Xy = 0.0, vapp = 0.0;
    unsigned long long W = 1ull << 32, dmask = 0;
    unsigned nev = 0, nsca = 0, nsurf = 0, fate = 0;
    ++st_launch;
#ifdef PDV_DEBUG
    if (sd.debug_check && ip == 0)                  // PDV_TEST_DEBUG_CHECK
      (void)PDV_IN((long long)sd.n_snap * row, (long long)sd.n_snap * row, PDV_DEBUG_SITE_SELFTEST);
    unsigned n_vtx = 0;
    const double tt = sd.t_trace;
    trace_put(sd, ip, n_vtx, x0, y0, sd.z_probe, 0.0, ux, uy, uz, 0, 0u);
#endif
    for (unsigned k = 1; fate == 0; ++k) {
      r = philox4x32_10(make_uint4((unsigned)pk, (unsigned)(pk >> 32), k, sd.stream_id), key);
      const double tau = -log(u23d(r.x));
      double Sn = S, vn = vcur;
      int what;
      if (fabs(uz) < 1e-9) {
        what = 3;
        double dvds;
        if (sd.expo) {                    // Eq. 20: dv/dS = (v_fs / beta) E / (1 - S E)
          dvds = sd.vb_d * sd.E_d / (1.0 - S * sd.E_d);
        } else {
          const int j = search_mass_d(sd.Sd, sd.n_v, S);
          dvds = sd.dv / (PDV_LD(sd.Sd, j + 1, sd.n_v + 1, PDV_DEBUG_SITE_MASS_NODE) -
                          PDV_LD(sd.Sd, j, sd.n_v + 1, PDV_DEBUG_SITE_MASS_NODE));
        }
        Xx += ux * tau * sd.inv_tau * dvds;
        Xy += uy * tau * sd.inv_tau * dvds;
      } else {
        Sn = S + tau * uz * sd.inv_tau;
        what = Sn >= 1.0 ? 1 : (Sn <= 0.0 ? 2 : 0);
      }
      if (what == 1) {
        Xx += ux / uz * (sd.v_top - vcur);
        Xy += uy / uz * (sd.v_top - vcur);
        if (sd.cone_all || uz >= sd.cos_alpha) {
          const double ax = x0 + ux / uz * sd.z_probe, ay = y0 + uy / uz * sd.z_probe;
          const double bx = Xx - ux / uz * sd.v_top, by = Xy - uy / uz * sd.v_top;
          const double fb = floor((vapp - sd.v_lo) * sd.inv_dbin);
          const int idx = fb < 0.0 ? 0 : (fb >= (double)n_bins ? n_bins + 1 : (int)fb + 1);
          for (int s = 0; s < sd.n_snap; ++s) {
            const double t = sd.t_snap[s];
            const double dx = ax + t * bx, dy = ay + t * by;
            if (sd.ap_all || dx * dx + dy * dy <= sd.r_ap2) {
              const long long n_h = (long long)sd.n_snap * row;
              if (PDV_IN((long long)s * row + idx, n_h, PDV_DEBUG_SITE_HISTOGRAM))
                atomicAdd(&sd.hist[(size_t)s * row + idx], W);
              if (PDV_IN((long long)s * row + n_bins + 2, n_h, PDV_DEBUG_SITE_HISTOGRAM))
                atomicAdd(&sd.hist[(size_t)s * row + n_bins + 2], 1ull);
              if (s < 64) dmask |= 1ull << s;
            }
          }
        }
#ifdef PDV_DEBUG
        trace_put(sd, ip, n_vtx, x0 + tt * Xx + ux / uz * (sd.z_probe - sd.v_top * tt),
                  y0 + tt * Xy + uy / uz * (sd.z_probe - sd.v_top * tt), sd.z_probe, 0.0, ux, uy, uz,
                  3, k);
#endif
        atomicAdd(&s_cnt[C_ESCAPES], 1ull);
        atomicAdd(&s_cnt[C_W_ESCAPED], W);
        fate = 1;
      } else if (what == 2) {
        Xx += ux / uz * (sd.v_fs - vcur);
        Xy += uy / uz * (sd.v_fs - vcur);
        S = 0.0;
        vcur = sd.v_fs;
        ++nev; ++nsurf; ++st_events; ++st_surf;
        const unsigned long long Wn =
            sd.R_q >= (1ull << 32) ? W : ((W * sd.R_q + (1ull << 31)) >> 32);
        if (Wn != W) atomicAdd(&s_cnt[C_W_ABS_SURFACE], W - Wn);
        W = Wn;
        const double uz_old = uz;
        if (sd.surface_mode == PDV_SURFACE_SPECULAR) {
          uz = -uz;
        } else {
          double ct, st;
          if (sd.surface_mode == PDV_SURFACE_LAMBERT) {
            const double a = u23d(r.y);
            ct = sqrt(a);
            st = sqrt(1.0 - a);
          } else {
            const double th = 0.5 * pi * u23d(r.y);
            ct = cos(th);
            st = sin(th);
          }
          const double ph = 2.0 * pi * u23d(r.z);
          ux = st * cos(ph);
          uy = st * sin(ph);
          uz = ct;
        }
        vapp += 0.5 * (uz - uz_old) * sd.v_fs;
        if (W == 0) fate = 3;
#ifdef PDV_DEBUG
        trace_put(sd, ip, n_vtx, x0 + tt * Xx, y0 + tt * Xy, sd.v_fs * tt, sd.v_fs, ux, uy, uz, 2, k);
#endif
      } else {
        if (what == 0 && sd.expo) {
          // Eq. 20 inverted in closed form: v = v_fs (1 - ln(1 - S E) / beta)
          vn = sd.v_fs - sd.vb_d * log1p(-Sn * sd.E_d);
          Xx += ux / uz * (vn - vcur);
          Xy += uy / uz * (vn - vcur);
        } else if (what == 0) {
          const int j = search_mass_d(sd.Sd, sd.n_v, Sn);
          const double s0 = PDV_LD(sd.Sd, j, sd.n_v + 1, PDV_DEBUG_SITE_MASS_NODE);
          const double s1 = PDV_LD(sd.Sd, j + 1, sd.n_v + 1, PDV_DEBUG_SITE_MASS_NODE);
          vn = sd.v_bot + j * sd.dv + (Sn - s0) / (s1 - s0) * sd.dv;
          Xx += ux / uz * (vn - vcur);
          Xy += uy / uz * (vn - vcur);
        }
        S = Sn;
        vcur = vn;
        ++nev; ++st_events;
        bool scatter;
        if (!sd.implicit) {
          scatter = (r.y >> 8) < sd.omega_q;               // Eq. 11
          if (!scatter) {
            atomicAdd(&s_cnt[C_W_ABS_PARTICLE], W);
            fate = 2;
          }
        } else {
          // implicit capture with the roulette on r1 (as in the FP32 kernel)
          const unsigned long long Wn = (W * sd.omega_q + (1ull << 23)) >> 24;
          if (W != Wn) atomicAdd(&s_cnt[C_W_ABS_PARTICLE], W - Wn);
          W = Wn;
          scatter = true;
          if (Wn < PDV_ROULETTE_W) {
            if (Wn != 0 && (r.y >> 8) < PDV_ROULETTE_Q) {
              atomicAdd(&s_cnt[C_W_RR_GAINED], (PDV_ROULETTE_M - 1) * Wn);
              W = Wn * PDV_ROULETTE_M;
            } else {
              atomicAdd(&s_cnt[C_W_RR_DROPPED], Wn);
              fate = 5;
              scatter = false;
            }
          }
        }
        if (scatter) {
          const unsigned m2 = r.z >> 8;
          int lo = 0, hi = sd.n_p - 2;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (PDV_LD(sd.Cq, mid, sd.n_p, PDV_DEBUG_SITE_PHASE_NODE) <= m2) lo = mid; else hi = mid - 1;
          }
          const unsigned c0 = PDV_LD(sd.Cq, lo, sd.n_p, PDV_DEBUG_SITE_PHASE_NODE);
          const unsigned c1 = PDV_LD(sd.Cq, lo + 1, sd.n_p, PDV_DEBUG_SITE_PHASE_NODE);
          const double th0 = PDV_LD(sd.th_d, lo, sd.n_p, PDV_DEBUG_SITE_PHASE_NODE);
          const double th1 = PDV_LD(sd.th_d, lo + 1, sd.n_p, PDV_DEBUG_SITE_PHASE_NODE);
          const double th = th0 + ((double)(m2 - c0) + 0.5) / (double)(c1 - c0) * (th1 - th0);
          const double ph = 2.0 * pi * u23d(r.w);
          const double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
          double nx, ny, nz;
          const double h2 = ux * ux + uy * uy;
          if (h2 < 1e-30) {                      // Eq. 17: vertical
            nx = st * cp; ny = st * sp; nz = uz >= 0.0 ? ct : -ct;
          } else {                               // Eq. 16, horizontal norm from (u_x, u_y)
            const double s = sqrt(h2);
            nx = st * (ux * uz * cp - uy * sp) / s + ux * ct;
            ny = st * (uy * uz * cp + ux * sp) / s + uy * ct;
            nz = -st * cp * s + uz * ct;
          }
          const double nn = sqrt(nx * nx + ny * ny + nz * nz);
          nx /= nn; ny /= nn; nz /= nn;
          vapp += 0.5 * (nz - uz) * vn;
          ux = nx; uy = ny; uz = nz;
          ++nsca; ++st_scat;
        }
#ifdef PDV_DEBUG
        trace_put(sd, ip, n_vtx, x0 + tt * Xx, y0 + tt * Xy, vn * tt, vn, ux, uy, uz, scatter ? 1 : 4,
                  k);
#endif
      }
      if (fate == 0 && nev >= sd.max_events) {
        atomicAdd(&s_cnt[C_W_TRUNCATED], W);
        atomicAdd(&s_cnt[C_TRUNCATED], 1ull);
        fate = 4;
      }
    }
    if (sd.packets) {
      pdv_packet_record rec;
      rec.n_events = nev;
      rec.n_scatters = nsca;
      rec.n_surface = nsurf;
      rec.fate = fate;
      rec.weight = W;
      rec.v_app = vapp;
      rec.detect_mask = dmask;
      if (PDV_IN(ip, sd.n_packets, PDV_DEBUG_SITE_PACKET)) sd.packets[ip] = rec;
    }
  }
  atomicAdd(&s_cnt[C_LAUNCHED], st_launch);
  atomicAdd(&s_cnt[C_EVENTS], st_events);
  atomicAdd(&s_cnt[C_SCATTERS], st_scat);
  atomicAdd(&s_cnt[C_SURFACE_HITS], st_surf);
  __syncthreads();
  if (threadIdx.x < C_NCOUNT && s_cnt[threadIdx.x]) atomicAdd(&sd.cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

void launch_transport_f64(const SetDesc* d_set, int grid, int block, cudaStream_t st) {
  k_transport_f64<<<grid, block, 0, st>>>(d_set);
}

// ------------------------------------------------------------------ Eq. 19
// One block per (snapshot, set): spectrum = weight / (2^32 N) (optionally per
// m/s), raw tallies and the per-snapshot counters.
__global__ void k_normalise(const SetDesc* __restrict__ sets, double* const* spec,
                            pdv_counters* const* cnt_out, unsigned long long* const* raw,
                            const unsigned* flags) {
  const SetDesc& sd = sets[blockIdx.y];
  const int s = blockIdx.x;
  if (s >= sd.n_snap) return;
  const int n_bins = sd.n_bins, row = hist_row(n_bins);
  // unlimited aperture: every time's tallies are those of row 0
  if (!PDV_IN((long long)(sd.ap_all ? 0 : s) * row + row - 1, (long long)sd.n_snap * row,
              PDV_DEBUG_SITE_HISTOGRAM))
    return;
  const unsigned long long* h = sd.hist + (size_t)(sd.ap_all ? 0 : s) * row;
  double scale = 1.0 / (kTwo32 * (double)sd.norm_packets);
  if (flags[blockIdx.y] & PDV_PER_DV) scale *= sd.inv_dbin;
  double* out = spec[blockIdx.y] + (size_t)s * n_bins;
  unsigned long long* rw = raw[blockIdx.y];
  unsigned long long part = 0;
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
    const unsigned long long v = h[b + 1];
    out[b] = (double)v * scale;
    part += v;
  }
  if (rw) {
    for (int b = threadIdx.x; b < n_bins + 2; b += blockDim.x) rw[(size_t)s * (n_bins + 2) + b] = h[b];
  }
  __shared__ unsigned long long red[32];
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long wdet = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) wdet += red[i];
    pdv_counters* co = cnt_out[blockIdx.y];
    if (co) {
      pdv_counters c;
      c.launched = sd.cnt[C_LAUNCHED];
      c.events = sd.cnt[C_EVENTS];
      c.scatters = sd.cnt[C_SCATTERS];
      c.surface_hits = sd.cnt[C_SURFACE_HITS];
      c.escapes = sd.cnt[C_ESCAPES];
      c.detected = h[n_bins + 2];
      c.w_detected = wdet;
      c.w_under = h[0];
      c.w_over = h[n_bins + 1];
      c.w_escaped_undetected = sd.cnt[C_W_ESCAPED] - wdet - h[0] - h[n_bins + 1];
      c.w_absorbed_particle = sd.cnt[C_W_ABS_PARTICLE];
      c.w_absorbed_surface = sd.cnt[C_W_ABS_SURFACE];
      c.w_truncated = sd.cnt[C_W_TRUNCATED];
      c.truncated = sd.cnt[C_TRUNCATED];
      c.w_roulette_dropped = sd.cnt[C_W_RR_DROPPED];
      c.w_roulette_gained = sd.cnt[C_W_RR_GAINED];
      co[s] = c;
    }
  }
}

cudaError_t transport_debug_io(DebugWord* out, bool reset, cudaStream_t st) {
#ifdef PDV_DEBUG
  return debug_word_io(out, reset, st);
#else
  (void)reset;
  (void)st;
  *out = DebugWord{};
  return cudaSuccess;
#endif
}

void launch_normalise(const SetDesc* d_sets, int n_sets, double* const* d_spec,
                      pdv_counters* const* d_cnt_out, unsigned long long* const* d_raw,
                      const unsigned* flags, int max_snap, cudaStream_t st) {
  k_normalise<<<dim3(max_snap, n_sets), 256, 0, st>>>(d_sets, d_spec, d_cnt_out, d_raw, flags);
}

}  // namespace pdv
