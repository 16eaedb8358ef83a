/*
 * pdv.h — C ABI of libpdv: GB300-native Monte Carlo simulation of the photon
 * Doppler velocimetry (PDV) spectrum of a shock-ejected particle cloud in
 * vacuum (Shi et al., "Reconstruction and interpretation of photon Doppler
 * velocimetry spectrum for ejecta particles from shock-loaded sample in
 * vacuum", arXiv:2012.00963, Section II).
 *
 * Conventions
 *  - Every function returns pdv_status: 0 on success, a negative code on
 *    error. pdv_last_error() returns a message for the calling thread's last
 *    error (valid until that thread's next failing call).
 *  - Host arrays passed in are caller-owned and copied during the call.
 *  - Device objects (contexts, clouds, tables) are library-owned and are
 *    released by the matching destroy function.
 *  - Output buffers are caller-owned: host memory by default, device memory
 *    when the request sets PDV_OUT_DEVICE. Device outputs are written on the
 *    context's stream; work that prepares them on another stream (for
 *    example a zero-fill) must be ordered before the call by the caller.
 *  - Units at the ABI follow the paper: area mass mg/cm^2, diameter um,
 *    wavelength nm, probe lengths mm, snapshot times us, velocities m/s.
 *  - Nothing here needs a particular framework: streams are plain
 *    cudaStream_t values passed as void*.
 */
#ifndef PDV_H
#define PDV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdv_ctx pdv_ctx;
typedef struct pdv_cloud pdv_cloud;
typedef uint64_t pdv_ticket;

typedef enum {
  PDV_OK = 0,
  PDV_EINVAL = -1,       /* invalid argument (message in pdv_last_error)      */
  PDV_ENOMEM = -2,       /* device or host allocation failed                  */
  PDV_ECUDA = -3,        /* a CUDA call failed                                 */
  PDV_EAGAIN = -4,       /* admission refused: not enough device memory/slots */
  PDV_ENOTREADY = -5,    /* request still running (pdv_poll)                  */
  PDV_ETIMEOUT = -6,     /* a bounded wait ran out                            */
  PDV_ECANCELLED = -7,   /* request cancelled                                 */
  PDV_EDEBUG = -8        /* libpdv_debug.so only: an index check failed during
                            the call; the access was skipped (pdv_debug_get)  */
} pdv_status;

enum { PDV_SURFACE_UNIFORM_THETA = 0, PDV_SURFACE_LAMBERT = 1, PDV_SURFACE_SPECULAR = 2 };
enum { PDV_PROFILE_EXPONENTIAL = 0, PDV_PROFILE_TABULATED = 1 };
enum { PDV_PREC_FP32 = 0, PDV_PREC_FP64 = 1 };

/* request flags */
#define PDV_OUT_DEVICE 0x1u   /* out_* pointers are device pointers            */
#define PDV_PER_DV     0x2u   /* spectrum divided by the bin width (per m/s)   */
#define PDV_IN_DEVICE  0x4u   /* input arrays are device pointers (pdv_ss_spectrum,
                                 pdv_extract_peaks)                            */
#define PDV_EXTRACT_SIMT 0x40u /* pdv_extract_peaks: both products as FP32 FMAs on the
                                 CUDA cores instead of the tensor cores         */
/* Implicit capture with Russian roulette, in place of the analog absorption
 * of Eq. 11 (Section II.B step (4)); off by default, exact free paths only
 * (n_layers == 0), both precisions. At every particle interaction the packet
 * scatters and keeps W' = floor((W omega_q + 2^23) / 2^24) of its weight
 * (omega_q = round(omega 2^24)); W - W' is absorbed by the particle. If
 * W' < PDV_ROULETTE_W the packet survives when (r1 >> 8) < PDV_ROULETTE_Q
 * (probability 1/16) with weight 16 W', else (and always when W' = 0) it is
 * dropped (fate 5). The expectation of every tally is that of the analog
 * scheme. */
#define PDV_IMPLICIT_CAPTURE 0x8u
#define PDV_ROULETTE_W (1ull << 22)  /* threshold, 2^32 fixed point (2^-10) */
#define PDV_ROULETTE_Q (1u << 20)    /* survival bound on r1 >> 8 (1/16)   */
#define PDV_ROULETTE_M 16u           /* survivor's weight factor           */

/* Test hook for the horizontal-flight rule: every packet enters at the top of
 * the cloud moving along +x, u = (1, 0, 0), instead of along -z. A flight with
 * |u_z| < 1e-9 keeps its height and runs tau* / mu(z) sideways, where mu is the
 * extinction per unit length at that height; the paper is silent on this case,
 * and random directions reach it with a probability of about 1e-9, so this flag
 * is how tests exercise it. Exact free paths only (n_layers == 0). */
#define PDV_TEST_HORIZONTAL_LAUNCH 0x10u

/* Test hook of the debug build (libpdv_debug.so, compiled with PDV_DEBUG):
 * the transport evaluates one index check at one past the end of the
 * request's histogram, without the access, so the call returns PDV_EDEBUG
 * with a record at PDV_DEBUG_SITE_SELFTEST. The release library refuses the
 * flag (PDV_EINVAL). */
#define PDV_TEST_DEBUG_CHECK 0x20u

/* Optional device allocator (NULL: cudaMallocAsync/cudaFreeAsync on the
 * context stream). Both callbacks are called from library threads. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, void* stream, void* user);
  void* user;
} pdv_allocator;

/* Particle cloud (Section II.C). Velocity profile: Eq. 20 (exponential law,
 * truncated at v_max and renormalised) or a tabulated, piecewise-linear
 * dm/dv > 0 on [prof_v[0], prof_v[n-1]] with prof_v[0] >= v_fs. Particles
 * fly freely, z = v t. Sizes: number log-normal of Eq. 21 (sigma_ln = 0 for a
 * single size); only the Sauter mean d_m exp(2.5 sigma^2) enters the optical
 * depth (Eq. 10). */
typedef struct {
  double rho_kg_m3;            /* particle density                       */
  double area_mass_mg_cm2;     /* total area mass m0 (0 = empty cloud)   */
  double v_fs;                 /* free-surface velocity, m/s             */
  double reflectivity;         /* free-surface reflectivity in [0, 1]    */
  int surface_mode;            /* PDV_SURFACE_*                          */
  int profile_kind;            /* PDV_PROFILE_*                          */
  double beta;                 /* Eq. 20 coefficient                     */
  double v_max;                /* m/s; 0: v_fs (1 + ln(1e6) / beta)      */
  const double* prof_v;        /* tabulated velocities (host)            */
  const double* prof_dmdv;     /* tabulated dm/dv (host, any scale)      */
  int prof_n;
  double d_median_um;          /* Eq. 21 median diameter                 */
  double sigma_ln;             /* Eq. 21 width                           */
  double wavelength_nm;        /* probe laser wavelength                 */
  int table_nodes;             /* velocity nodes of the mass table (0 = 2048, max 16384) */
} pdv_cloud_desc;

/* Probe geometry: a collimated beam of radius beam_radius_mm launched along
 * -z from the plane z = z_probe_mm; detection on the same plane within
 * aperture_radius_mm (<= 0: unlimited) and within cone_half_angle_rad of +z
 * (>= pi/2: every upward packet). Eq. 6 boundary conditions. */
typedef struct {
  double z_probe_mm;
  double beam_radius_mm;
  double aperture_radius_mm;
  double cone_half_angle_rad;
} pdv_probe;

/* Per-snapshot tallies. Weights are 2^32 fixed point per launched packet;
 * w_detected + w_under + w_over + w_escaped_undetected + w_absorbed_particle
 * + w_absorbed_surface + w_truncated + w_roulette_dropped
 * == launched * 2^32 + w_roulette_gained exactly (the last two are 0 unless
 * PDV_IMPLICIT_CAPTURE is set: the weight of dropped packets, and the
 * weight that survivors gained, (PDV_ROULETTE_M - 1) W' each). */
typedef struct {
  uint64_t launched, events, scatters, surface_hits, escapes, detected;
  uint64_t w_detected, w_under, w_over, w_escaped_undetected;
  uint64_t w_absorbed_particle, w_absorbed_surface, w_truncated, truncated;
  uint64_t w_roulette_dropped, w_roulette_gained;
} pdv_counters;

/* Per-packet record (debug / parity dumps; snapshot 0 unless stated). */
typedef struct {
  uint32_t n_events, n_scatters, n_surface, fate;  /* fate: 1 escaped, 2 absorbed by a particle, 3 absorbed at the surface, 4 truncated, 5 dropped by the roulette */
  uint64_t weight;                                 /* weight when the fate was decided, 2^32 fixed point */
  double v_app;                                    /* apparent velocity, m/s */
  uint64_t detect_mask;                            /* bit s: detected at snapshot s < 64 */
} pdv_packet_record;

/* One spectrum request: packets [packet_begin, packet_begin + n_packets)
 * of the stream (seed, stream_id), tallied at every snapshot time into
 * n_bins bins over [v_lo, v_hi). Output spectrum[s * n_bins + b] =
 * sum of detected weights / (2^32 n_packets) (Eq. 19 without the
 * sqrt(I0/n0) scale). Packet ranges of one stream add up exactly: raw
 * tallies of [0, k) and [k, N) sum to those of [0, N). */
typedef struct {
  const pdv_cloud* cloud;
  pdv_probe probe;
  const double* t_snap_us;         /* host array [n_snap], each > 0      */
  int n_snap;                      /* 1..4096                            */
  uint64_t n_packets;              /* >= 1, <= 4e9                       */
  uint64_t packet_begin;
  uint64_t seed;
  uint32_t stream_id;
  uint32_t max_events;             /* per packet; 0 = 1e6; 2^32-1 acts as 2^32-2 */
  int n_bins;                      /* 1..65536                           */
  double v_lo, v_hi;               /* m/s, v_hi > v_lo                   */
  int precision;                   /* PDV_PREC_FP32 | PDV_PREC_FP64      */
  uint32_t flags;                  /* PDV_OUT_DEVICE | PDV_PER_DV | PDV_IMPLICIT_CAPTURE
                                      | PDV_TEST_HORIZONTAL_LAUNCH */
  double* out_spectrum;            /* [n_snap * n_bins], required        */
  uint64_t* out_raw;               /* optional [n_snap * (n_bins + 2)]: under, bins, over */
  pdv_counters* out_counters;      /* optional [n_snap]                  */
  pdv_packet_record* out_packets;  /* optional [n_packets] (n_packets <= 2^26) */
  uint32_t n_layers;               /* 0: exact free paths (the default). > 0: the
                                      paper's own scheme (Section II.B steps (2)-(6)):
                                      synchronous steps of (v_max - v_fs) t / n_layers,
                                      a Bernoulli pass per layer with Eq. 7 / Eq. 10,
                                      the interaction at the step's end, and the polar
                                      angle by acceptance-rejection over the sphere
                                      (p(theta) / max p). FP32 only, through
                                      pdv_simulate_spectrum; max_events then bounds
                                      the steps. The paper uses 1000.        */
  uint32_t reserved;               /* 0                                   */
} pdv_request;

/* Launch parameters of the persistent FP32 kernel (pdv_autotune picks them). */
typedef struct {
  int block_threads;               /* 128, 256, 512 (0 = 256)            */
  int blocks_per_sm;               /* 0 = occupancy maximum              */
  int tile_packets;                /* packets a warp claims at a time from its
                                      request's counter: 0 (64) or 16..65536 */
  int hist_mode;                   /* 0 auto, 1 global atomics, 2 shared-memory privatised */
} pdv_tuning;

typedef struct {
  double tau_tot;                  /* optical depth of the cloud (Eq. 10) */
  double v_bot, v_top;             /* velocity span of the cloud, m/s     */
  double d_sauter_um;              /* d_m exp(2.5 sigma^2)                */
  double g_table;                  /* mean cosine of the sampled phase law */
  double q_ext, albedo;
  int table_nodes;
  int has_phase;
} pdv_cloud_info;

typedef struct {
  uint64_t kernel_launches;        /* kernels this context has launched   */
  double last_transport_ms;        /* CUDA-event time of the last transport kernel */
  uint64_t last_events;            /* events of the last synchronous call */
  int transport_grid, transport_block;
  double last_model_ms;            /* CUDA-event time of the last pdv_ss_spectrum /
                                      pdv_extract_peaks main kernel      */
  uint64_t last_steps;             /* layer steps of the last layer-stepping call */
  int32_t transport_fast;          /* 1: the last FP32 transport launch ran the build for
                                      the common set configuration (exponential law, phase
                                      angles from the node table, vertical launch, uniform-
                                      angle wall with R < 1, no packet records) on every
                                      set; 0: the generic build, or not an FP32 launch
                                      (the serving thread's launches do not set it) */
  int32_t reserved;
} pdv_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on `device`. cuda_stream: a cudaStream_t to run on (NULL:
 * the library creates its own non-blocking stream). alloc: optional device
 * allocator. On error *out is NULL. */
pdv_status pdv_ctx_create(int device, void* cuda_stream, const pdv_allocator* alloc,
                          pdv_ctx** out);
/* Waits for the context's work, stops the serving thread, frees everything.
 * Destroy every cloud made on the context (pdv_destroy_cloud) first: device
 * memory comes from the context's own stream-ordered pool, which keeps up to
 * 2 GiB of freed memory mapped between calls and is released here. */
pdv_status pdv_ctx_destroy(pdv_ctx* ctx);
const char* pdv_last_error(void);
pdv_status pdv_get_stats(pdv_ctx* ctx, pdv_stats* out);
pdv_status pdv_set_tuning(pdv_ctx* ctx, const pdv_tuning* tuning);

/* ---------------------------------------------------------------- cloud */

/* Build the cloud's cumulative mass-fraction table on the device in FP64
 * (Eq. 20, z = v t). The cloud is usable once a phase table is set.
 * Errors: PDV_EINVAL (rho <= 0, m0 < 0, d_m <= 0, sigma < 0, R outside [0,1],
 * v_fs <= 0, v_max <= v_fs, bad tabulated profile), PDV_ENOMEM, PDV_ECUDA. */
pdv_status pdv_create_cloud(pdv_ctx* ctx, const pdv_cloud_desc* desc, pdv_cloud** out);

/* Set the phase function p(theta) (Eq. 13, unnormalised, >= 0, theta strictly
 * increasing from 0 to pi, n in 2..65536), the size-averaged extinction
 * efficiency Q_ext (Eq. 10) and the single-scattering albedo K_sca/K_ext
 * (Eq. 11). Builds the integer inverse CDF on the device in FP64. */
pdv_status pdv_set_phase_table(pdv_cloud* cloud, int n, const double* theta_rad,
                               const double* p, double q_ext_eff, double albedo);
pdv_status pdv_cloud_get_info(const pdv_cloud* cloud, pdv_cloud_info* out);
pdv_status pdv_destroy_cloud(pdv_cloud* cloud);

/* Henyey–Greenstein p(theta) on n uniform angles over [0, pi] (host helper). */
pdv_status pdv_phase_hg(double g, int n, double* theta_rad, double* p);

/* Size-averaged Mie phase table (Eq. 12-14, Eq. 21) computed on the device in
 * FP64: theta_rad[n_angle] uniform over [0, pi], p[n_angle] proportional to
 * <|S1|^2 + |S2|^2>, Q_ext = <d^2 Q_ext>/<d^2>, albedo = <C_sca>/<C_ext>,
 * g = <C_sca g>/<C_sca>. Gauss–Legendre in ln d over ln d_m +- 6 sigma with
 * n_size nodes (sigma = 0: one size). Outputs are host arrays. Errors:
 * PDV_EINVAL (m_im < 0, sizes <= 0, n_angle < 2, size parameter > 20000). */
pdv_status pdv_mie_table(pdv_ctx* ctx, double m_re, double m_im, double wavelength_nm,
                         double d_median_um, double sigma_ln, int n_size, int n_angle,
                         double* theta_rad, double* p, double* q_ext_eff, double* albedo,
                         double* g);

/* ---------------------------------------------------------------- spectra */

/* Run one request to completion (blocking): transport all packets, tally,
 * normalise and copy the outputs. Errors: PDV_EINVAL (see pdv_request; also
 * a snapshot with the top of the cloud at or above the probe plane),
 * PDV_ENOMEM, PDV_ECUDA. */
pdv_status pdv_simulate_spectrum(pdv_ctx* ctx, const pdv_request* req);

/* Run n requests in one persistent launch (FP32 requests only; FP64 requests
 * run one after another), replayed from a captured CUDA graph cached per
 * batch shape. Outputs as for pdv_simulate_spectrum. */
pdv_status pdv_simulate_batch(pdv_ctx* ctx, const pdv_request* reqs, int n);

/* Time candidate launch parameters on a short version of the batch (1/16 of
 * each request's packets, at least 65536) and keep the fastest in the context
 * (and in *out if not NULL). The search covers block_threads {128, 256},
 * hist_mode {1, 2} (global or block-private histograms), blocks_per_sm
 * {0 (as many as fit), 2} and tile_packets {32, 64, 256}. With a cache file set
 * (pdv_set_autotune_cache), a choice already recorded there for this device
 * and batch shape is taken without timing, and a new choice is added to the
 * file. A deployment tool with no counterpart in the paper. */
pdv_status pdv_autotune(pdv_ctx* ctx, const pdv_request* reqs, int n, pdv_tuning* out);

/* Keep pdv_autotune's choices in a JSON file (NULL: no cache). The file maps
 * "device|sms|sets|packets|snapshots|bins|flags" keys, one per device name
 * and batch shape, to the chosen pdv_tuning fields. Errors: PDV_EINVAL. */
pdv_status pdv_set_autotune_cache(pdv_ctx* ctx, const char* path);

/* Measured instruction-issue rate of the context's GPU, the denominator of
 * the issue-rate roofline the transport kernels are reported against (their
 * work is integer and FP32 instruction issue, not a contraction or memory
 * traffic). Runs a kernel of independent FP32 fused multiply-adds, eight
 * chains per thread and 64 warps per SM, for about `seconds` (0 < seconds
 * <= 10) on the context's stream, waits for it, and writes FMA
 * thread-instructions per second to *out. The loop's own three instructions
 * per 64 FMAs are not counted, so the figure is a slight lower bound of the
 * issue rate at the clock the GPU ran. Errors: PDV_EINVAL (NULL arguments,
 * seconds out of range), PDV_ECUDA. */
pdv_status pdv_measure_issue_rate(pdv_ctx* ctx, double seconds, double* out);

/* The same FP32 spectrum as pdv_simulate_spectrum for callers that cannot
 * allocate device memory while they run (an allocator or memory plan that
 * forbids cudaMalloc after start-up). The paper has no counterpart: it is a
 * deployment variant. Its scratch is a fixed 4 MiB array in device memory that
 * every GPU loading the library keeps until the process exits. A request must
 * fit in it: 2048 + ceil256(8 n_snap (n_bins + 3)) + ceil256(24 n_snap) bytes
 * at most 4 MiB, where ceil256 rounds up to a multiple of 256 (roughly
 * n_snap (n_bins + 6) * 8 + 2.5 KiB), else PDV_EINVAL. Outputs must be device
 * buffers (PDV_OUT_DEVICE); precision must be FP32. The cloud's tables are
 * made beforehand by pdv_create_cloud and pdv_set_phase_table. pdv_ctx_create
 * does all the set-up this call needs: it looks the array's device address up
 * (which maps the array on the context's device), loads the kernels the call
 * launches and reserves host buffers for the snapshot times, so the call
 * itself allocates neither device nor host memory. Do not reset the device
 * (cudaDeviceReset) while a context lives. All calls share the array and it
 * keeps the last call's contents (cleared at the start of each call); calls
 * that overlap on the GPU race. Blocking. Errors: PDV_EINVAL, PDV_ECUDA. */
pdv_status pdv_simulate_spectrum_static(pdv_ctx* ctx, const pdv_request* req);

/* ---------------------------------------------------------------- serving */

/* Admit a request into the context's continuous-batching loop. The request's
 * cloud and output buffers must stay valid until pdv_poll reports completion.
 * Returns PDV_EAGAIN when device memory or request slots do not allow it now:
 * at most max_requests submitted requests may be held (running, or finished
 * and not yet returned by pdv_poll), and the request's device buffers must fit
 * in the device's free memory less reserve_bytes (pdv_set_serving_limits). */
pdv_status pdv_submit(pdv_ctx* ctx, const pdv_request* req, pdv_ticket* out);

/* Admission limits of pdv_submit: max_requests in [1, 65536] (default 1024)
 * and reserve_bytes of device memory kept free (default 256 MiB). A deployment
 * variant with no counterpart in the paper. Takes effect at the next submit.
 * Errors: PDV_EINVAL. */
pdv_status pdv_set_serving_limits(pdv_ctx* ctx, int max_requests, uint64_t reserve_bytes);

/* Wait up to timeout_us for a ticket: PDV_OK (done, outputs written, ticket
 * released), PDV_ENOTREADY (still running), or the request's error. */
pdv_status pdv_poll(pdv_ctx* ctx, pdv_ticket ticket, uint32_t timeout_us);

/* Cancel a queued or running request; its ticket then polls PDV_ECANCELLED. */
pdv_status pdv_cancel(pdv_ctx* ctx, pdv_ticket ticket);

/* ---------------------------------------------------------------- spectrum model
 *
 * Single-scattering spectrum (Section III.B, Eq. 22-28): light scattered once,
 * straight back, by the particles at velocity v, attenuated on the way in and
 * out by the mass above them. With f the mass density of Eq. 20 (unit area
 * mass; renormalised over [v_fs, v_max] when v_max is finite) and Fbar(v) the
 * mass fraction above v,
 *     I(v) = prefactor * tau0 * f(v) * exp(-tau0 * Fbar(v)),
 * which is Eq. 28 for the untruncated law (Fbar = f v_fs / beta). tau0 is the
 * optical thickness of Eq. 27 (extinction by back-scattering and absorption,
 * g_back K_ext of Eq. 25); prefactor holds the size factors of Eq. 28. */
typedef struct {
  double beta;                     /* velocity coefficient of Eq. 20, > 0            */
  double tau0;                     /* optical thickness of Eq. 27, >= 0              */
  double v_fs;                     /* free-surface velocity, m/s, > 0                */
  double v_max;                    /* cut of the law, m/s; <= v_fs or inf: untruncated */
  double prefactor;                /* constant factor of Eq. 28 (1 for the shape)    */
} pdv_ss_set;

/* Integrate the single-scattering spectrum of each set over n_bins uniform
 * bins of [v_lo, v_hi] (out[set * n_bins + bin], FP64 output computed in FP32
 * arithmetic from FP64 per-set constants; relative error about 1e-6 of the
 * spectrum's largest bin). The bin integral is exact through the antiderivative
 * prefactor * exp(-tau0 Fbar(v)). With PDV_PER_DV each bin is divided by its
 * width. sets: host array, or device array with PDV_IN_DEVICE (those sets are
 * checked on the device). out: host array, or device with PDV_OUT_DEVICE.
 * Errors: PDV_EINVAL (n_sets < 0, n_bins < 1, v_hi <= v_lo, a set with
 * beta <= 0, tau0 < 0 or v_fs <= 0: its bins are then NaN), PDV_ENOMEM,
 * PDV_ECUDA. */
pdv_status pdv_ss_spectrum(pdv_ctx* ctx, const pdv_ss_set* sets, int n_sets, int n_bins,
                           double v_lo, double v_hi, uint32_t flags, double* out);

/* ---------------------------------------------------------------- peak extraction
 *
 * Section III.C and Eq. 29-35: low-pass the binned spectrum with the real DFT
 * (modes 0..k_c kept), find the largest smoothed value on the bin centres
 * inside the search window, refine it by up to 8 Newton steps on the
 * analytic first derivative (each kept within one bin of the grid maximum),
 * and read off the relative curvature I''/I at the peak in x = v / v_fs:
 *     beta = sqrt(-I''/I)  (Eq. 34),  tau0 = exp(beta (x_peak - 1))  (Eq. 31). */
typedef struct {
  int k_c;                         /* modes kept, 1 <= k_c < n_bins / 2              */
  int reserved;
  double x_min, x_max;             /* search window in v / v_fs (bin centres inside
                                      it); -inf / +inf for the whole range          */
} pdv_peak_opts;

enum { PDV_PEAK_OK = 0, PDV_PEAK_NO_PEAK = 1, PDV_PEAK_NOT_MAX = 2, PDV_PEAK_EDGE = 3 };

typedef struct {
  double x_peak;                   /* peak position, v / v_fs                        */
  double i_peak;                   /* smoothed spectrum at the peak                  */
  double curvature;                /* I''/I at the peak, per (v / v_fs)^2            */
  double beta, tau0;               /* Eq. 35; NaN unless status is PDV_PEAK_OK       */
  int32_t status;                  /* PDV_PEAK_*                                     */
  int32_t j_max;                   /* bin of the smoothed grid maximum (-1: none)    */
} pdv_peak;

/* Extract the main peak of n_spectra spectra of n_bins uniform bins over
 * [v_lo, v_hi] (row-major [n_spectra][n_bins]). Arithmetic is FP32 with
 * cosine / sine tables computed in FP64 and rounded to FP32; inputs are
 * rounded to FP32 (magnitudes below 1.2e-38 flush to zero). For k_c <= 63
 * the two products (the DFT and the window values) run on the tensor cores:
 * TF32 operands split into a high and a low part, three products per step,
 * so each term carries at most about 2^-22 of |x| |F| of error, and the
 * truncating accumulators are summed in short runs and added in FP32. Larger
 * cut-offs, and every cut-off with PDV_EXTRACT_SIMT, run them as FP32 FMAs on
 * the CUDA cores. Accuracy: about 1e-6 relative in x_peak,
 * I''/I, beta and tau0 while the cut-off smooths
 * (k_c well below n_bins / 2); as k_c nears n_bins / 2 the
 * FP32 rounding of the input itself, amplified by up to pi^2 per bin in the
 * second derivative, dominates the curvature.
 * spectra: host array, or device with PDV_IN_DEVICE. out: host array,
 * or device with PDV_OUT_DEVICE. Errors: PDV_EINVAL (n_spectra < 0,
 * n_bins < 3 or > 8192, k_c outside [1, n_bins / 2), v_hi <= v_lo, v_fs <= 0),
 * PDV_ENOMEM, PDV_ECUDA, PDV_ETIMEOUT (a bounded wait of the tensor-core
 * kernel for its products ran out). */
pdv_status pdv_extract_peaks(pdv_ctx* ctx, const double* spectra, int n_spectra, int n_bins,
                             double v_lo, double v_hi, double v_fs, const pdv_peak_opts* opts,
                             uint32_t flags, pdv_peak* out);

/* ---------------------------------------------------------------- debug build
 *
 * libpdv_debug.so is the same library compiled with PDV_DEBUG. Its transport,
 * layer-stepping and normalisation kernels check every index into the staged
 * tables, the tallies and the per-packet outputs before the access. A failed
 * check skips the access and records itself in a device word; it never traps,
 * so the context stays usable. pdv_simulate_spectrum, pdv_simulate_batch and
 * pdv_simulate_spectrum_static read the word after their kernels finish and
 * return PDV_EDEBUG while it holds a failure (until pdv_debug_get resets it).
 * The release library (libpdv.so) compiles the checks out. */
enum {
  PDV_DEBUG_SITE_NONE = 0,
  PDV_DEBUG_SITE_MASS_GUIDE = 1,   /* guide of the velocity table            */
  PDV_DEBUG_SITE_MASS_NODE = 2,    /* velocity table nodes (S_j, slopes)     */
  PDV_DEBUG_SITE_PHASE_GUIDE = 3,  /* guide of the phase CDF                 */
  PDV_DEBUG_SITE_PHASE_NODE = 4,   /* phase CDF nodes, angles, (cos, sin)    */
  PDV_DEBUG_SITE_TURN = 5,         /* table of (cos, sin) of 2 pi j / 1024   */
  PDV_DEBUG_SITE_SNAPSHOT = 6,     /* snapshot times and their order         */
  PDV_DEBUG_SITE_HISTOGRAM = 7,    /* tally rows                             */
  PDV_DEBUG_SITE_PACKET = 8,       /* per-packet records                     */
  PDV_DEBUG_SITE_SELFTEST = 9      /* PDV_TEST_DEBUG_CHECK                   */
};

typedef struct {
  int32_t debug_build;             /* 1: libpdv_debug.so; 0: the release library
                                      (the other fields are then 0)          */
  uint32_t site;                   /* PDV_DEBUG_SITE_* of the first failed check */
  uint64_t violations;             /* failed checks since the last reset     */
  int64_t index;                   /* the first failed check: its index ...  */
  int64_t bound;                   /* ... and the size it was checked against */
} pdv_debug_info;

/* Read (and with reset != 0 clear) the failed-check record of the context's
 * device. Waits for the context's stream first. */
pdv_status pdv_debug_get(pdv_ctx* ctx, pdv_debug_info* out, int reset);

/* One vertex of a packet's path at the request's first snapshot time t
 * (Section II.B steps (1)-(6)): position (m), the velocity coordinate z / t
 * of the vertex (m/s; 0 at the probe plane), the direction after the vertex,
 * and what happened there: 0 launch at the probe plane, 1 particle scatter,
 * 2 free surface, 3 escape (at the probe plane), 4 absorbed by a particle or
 * dropped by the roulette. event: the Philox event counter of the vertex. */
typedef struct {
  double x, y, z, v, ux, uy, uz;
  int32_t kind;
  uint32_t event;
} pdv_trace_vertex;

/* libpdv_debug.so only (the release library returns PDV_EINVAL): the next
 * pdv_simulate_spectrum on this context that asks for per-packet records
 * (out_packets) also writes the paths of its first n_trace packets to
 * out[n_trace][max_vertices] (host), in FP32 or FP64 as the request's
 * precision; unused slots get kind -1. Exact free paths only (n_layers == 0).
 * n_trace in 1..65536, max_vertices in 1..4096; n_trace = 0 disarms. */
pdv_status pdv_debug_set_trace(pdv_ctx* ctx, int n_trace, int max_vertices,
                               pdv_trace_vertex* out);

#ifdef __cplusplus
}
#endif

#endif /* PDV_H */
