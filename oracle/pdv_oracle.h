/*
 * pdv_oracle.h — plain, slow FP64 CPU oracle for the Monte Carlo PDV spectrum
 * of a shock-ejected particle cloud in vacuum (Shi et al., arXiv:2012.00963,
 * Section II "Reconstruction of PDV spectrum").
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline / reference leg of the benchmark may load this library. The
 * product path (the CUDA library under paper_2012_00963_gb300/) never links,
 * loads or calls it, and this oracle shares no code with that library: it has
 * its own Philox generator, its own velocity-profile inversion, its own Mie
 * series and its own phase-function sampler.
 *
 * Every quantity is FP64. Each packet is transported separately for each
 * snapshot time (the plain definition); common random numbers across
 * snapshots come from the counter layout (packet, event), which holds no
 * snapshot index.
 *
 * Parity status per function:
 *   orc_philox4x32_10      pinned (published known-answer vectors)
 *   orc_profile_*          pinned (closed form / independent quadrature)
 *   orc_mie_single         pinned (Rayleigh limit, optical theorem, large-x
 *                          extinction paradox, real-index energy balance)
 *   orc_mie_table          pinned (phase normalisation, g from coefficients)
 *   orc_phase_cdf          pinned (sample mean cosine vs closed form, KS)
 *   orc_rotate             pinned (unit norm, scattering angle, azimuth mean)
 *   orc_simulate           pinned (Beer–Lambert, empty-cloud delta peak and
 *                          detected weight, exact backscatter sheet, weight
 *                          conservation, order-1 single-scattering integral,
 *                          time invariance, Doppler = -1/2 dL/dt);
 *                          the full multiple-scattering spectrum beyond those
 *                          invariants is "parity unpinned" (the paper prints
 *                          no spectrum values). Implicit capture is pinned
 *                          by the reductions omega = 1 (the analog walk) and
 *                          omega = 0 (the analog absorbed weight), the weight
 *                          law W = 2^32 omega^k 16^j of the k-scatter escapes,
 *                          its conservation identity and the analog means.
 *   v_app_spread           pinned (zero at zero perturbation, linear in the
 *                          perturbation size, zero for the exact specular
 *                          echo, thread-count invariant)
 */
#ifndef PDV_ORACLE_H
#define PDV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Counter slots, one row per snapshot (weights are 2^32 fixed point). */
enum {
  ORC_LAUNCHED = 0,      /* packets launched                                  */
  ORC_EVENTS,            /* particle interactions + free-surface reflections  */
  ORC_SCATTERS,          /* particle scatterings                              */
  ORC_SURFACE_HITS,      /* free-surface reflections                          */
  ORC_ESCAPES,           /* packets leaving through the top of the cloud      */
  ORC_DETECTED,          /* escaped packets inside the aperture and the cone  */
  ORC_W_DETECTED,        /* weight detected with v_app in [v_lo, v_hi)        */
  ORC_W_UNDER,           /* weight detected with v_app < v_lo                 */
  ORC_W_OVER,            /* weight detected with v_app >= v_hi                */
  ORC_W_ESC_UNDETECTED,  /* weight escaped outside the aperture or the cone   */
  ORC_W_ABS_PARTICLE,    /* weight absorbed by particles (Eq. 11)             */
  ORC_W_ABS_SURFACE,     /* weight absorbed by the free surface (1 - R)       */
  ORC_W_TRUNCATED,       /* weight of packets stopped by the event limit      */
  ORC_TRUNCATED,         /* packets stopped by the event limit                */
  ORC_W_RR_DROPPED,      /* implicit capture: weight dropped by the roulette  */
  ORC_W_RR_GAINED,       /* implicit capture: weight survivors gained         */
  ORC_NCOUNTERS
};

enum { ORC_FATE_ESCAPED = 1, ORC_FATE_ABS_PARTICLE = 2, ORC_FATE_ABS_SURFACE = 3,
       ORC_FATE_TRUNCATED = 4, ORC_FATE_DROPPED = 5 };

/* Implicit capture with Russian roulette (a variance-reduction variant of
 * Section II.B step (4); the paper itself uses the analog choice of Eq. 11):
 * the packet keeps round(W omega_q / 2^24) at each particle interaction and,
 * below ORC_RR_W, survives with probability 1/ORC_RR_M at ORC_RR_M times
 * its weight. */
#define ORC_RR_W ((uint64_t)1 << 22)   /* threshold, 2^32 fixed point      */
#define ORC_RR_M 16u                   /* survival 1 in 16, weight x 16    */

#define ORC_NORDER 5   /* scattering-order histograms: orders 0..3 and 4+ */

typedef struct {
  /* cloud: Eq. 8-10, Eq. 20-21 */
  double rho;            /* particle material density, kg/m^3                */
  double m0;             /* total area mass, kg/m^2                          */
  double v_fs;           /* free-surface velocity, m/s                       */
  double reflectivity;   /* free-surface reflectivity R in [0, 1]            */
  int surface_mode;      /* 0 uniform polar angle, 1 Lambertian, 2 specular  */
  int profile_kind;      /* 0 exponential (Eq. 20), 1 tabulated dm/dv        */
  double beta;           /* Eq. 20 velocity coefficient                      */
  double v_max;          /* top of the cloud for the exponential law, m/s    */
  const double* prof_v;  /* tabulated: velocities, strictly increasing, m/s  */
  const double* prof_f;  /* tabulated: dm/dv (> 0), any scale                */
  int prof_n;
  double d_m;            /* median diameter, m (Eq. 21)                      */
  double sigma_ln;       /* log-normal width (0 = monodisperse)              */
  double q_ext;          /* area-weighted mean extinction efficiency         */
  double albedo;         /* single-scattering albedo K_sca/K_ext (Eq. 11)    */
  /* phase function table: theta strictly increasing from 0 to pi */
  int n_phase;
  const double* theta;
  const double* p;       /* unnormalised p(theta) >= 0                       */
  /* probe */
  double z_probe;        /* probe plane height above the sample origin, m    */
  double r_beam;         /* beam radius, m                                   */
  double r_ap;           /* aperture radius, m; <= 0 means unlimited         */
  double cone_alpha;     /* acceptance half angle, rad; >= pi/2 = all upward */
  /* snapshots and tally */
  int n_snap;
  const double* t_snap;  /* snapshot times, s                                */
  int n_bins;
  double v_lo, v_hi;     /* apparent-velocity histogram range, m/s           */
  /* packets */
  uint64_t packet_begin; /* first packet index                               */
  uint64_t n_packets;
  uint64_t seed;
  uint32_t stream_id;
  uint32_t max_events;   /* event limit per packet (0 = 1000000); with layer
                            stepping it bounds the steps                       */
  uint32_t n_layers;     /* 0: exact free paths; > 0: the paper's synchronous
                            stepping, H / n_layers per step (Section II.B)     */
  uint32_t implicit_capture; /* 1: implicit capture + roulette (exact free
                            paths only); 0: the analog choice of Eq. 11        */
  /* Rounding sensitivity of each packet's v_app (test support, only with a
   * packets array): spread_runs perturbed FP64 re-runs of snapshot 0 in which
   * every flight's optical length, every new direction and every stored
   * direction component carry a random error the size of a binary32 rounding
   * (standard deviations in units of u = 2^-24). 0 runs: none. */
  uint32_t test_horizontal_launch; /* 1: packets enter moving along +x (a test
                            of the horizontal-flight rule; exact paths only)   */
  uint32_t spread_runs;
  double spread_flight;  /* relative, per flight                             */
  double spread_turn;    /* absolute, per direction component at each turn   */
  double spread_store;   /* relative, per stored direction component         */
} orc_problem;

typedef struct {
  uint32_t n_events, n_scatters, n_surface, fate;
  uint64_t weight;       /* final weight (2^32 fixed point)                  */
  double v_app;          /* apparent velocity accumulated (snapshot 0)       */
  uint64_t detect_mask;  /* bit s: detected at snapshot s (s < 64)           */
  double v_app_spread;   /* largest |v_app' - v_app| over the perturbed re-runs
                            that kept the event count (0 without re-runs)      */
  uint32_t n_unstable;   /* perturbed re-runs whose event count changed      */
  uint32_t pad_;
} orc_packet;

typedef struct {
  double x, y, z;        /* vertex position, m                               */
  double v;              /* velocity of the reflecting particle / surface    */
  double ux, uy, uz;     /* direction after the vertex                       */
  int kind;              /* 0 launch, 1 scatter, 2 surface, 3 escape (probe) */
} orc_vertex;

/* Derived cloud constants. Returns 0 on success, -1 on invalid input. */
int orc_cloud_constants(const orc_problem* pb, double* tau_tot, double* v_bot,
                        double* v_top, double* d_sauter);

/* Cumulative mass fraction s(v) in [0, 1] and its inverse v(s). */
double orc_profile_cdf(const orc_problem* pb, double v);
double orc_profile_inverse(const orc_problem* pb, double s);

/* Philox4x32-10 block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Mie series for one sphere: size parameter x, relative index m = mr + i mi.
 * Fills q[0..3] = (Q_ext, Q_sca, Q_back, g) and, if n_mu > 0, |S1|^2 and
 * |S2|^2 at mu[] (cos theta), plus S(0) real/imag in s0[0..1]. Returns the
 * number of series terms. */
int orc_mie_single(double x, double mr, double mi, int n_mu, const double* mu,
                   double* s11, double* s22, double* q, double* s0);

/* Size-averaged Mie phase table for a number-log-normal distribution. */
int orc_mie_table(double mr, double mi, double wavelength, double d_m, double sigma_ln,
                  int n_size, int n_angle, double* theta, double* p,
                  double* q_ext, double* albedo, double* g);

/* Henyey–Greenstein p(theta) on a uniform grid of n angles over [0, pi]. */
void orc_hg_table(double g, int n, double* theta, double* p);

/* Integer phase CDF C_q (2^24 scale) and the mean cosine of the sampled law. */
int orc_phase_cdf(int n, const double* theta, const double* p, uint32_t* cq, double* g_tab);

/* Scattering angle sampled from C_q with the 24-bit integer m. */
double orc_phase_sample(int n, const double* theta, const uint32_t* cq, uint32_t m);

/* Direction rotation by (theta, phi), Eq. 16-17, renormalised. */
void orc_rotate(double u[3], double cos_t, double sin_t, double cos_p, double sin_p);

/* cos(theta) drawn by the layer-stepping scheme's acceptance-rejection for
 * packet pk at step `step` (uses seed, stream_id and the phase table of pb). */
double orc_phase_ar_cos(const orc_problem* pb, uint64_t pk, uint32_t step);

/* Full simulation. hist: [n_snap][n_bins]; counters: [n_snap][ORC_NCOUNTERS];
 * order_hist (optional): [n_snap][ORC_NORDER][n_bins]; packets (optional):
 * [n_packets]; trace (optional): [n_trace][max_vertices] for the first
 * n_trace packets at snapshot 0, unused slots get kind = -1.
 * Returns 0, or -1 on invalid input. */
int orc_simulate(const orc_problem* pb, int n_threads, uint64_t* hist, uint64_t* counters,
                 uint64_t* order_hist, orc_packet* packets, int n_trace, int max_vertices,
                 orc_vertex* trace);

#ifdef __cplusplus
}
#endif
#endif
