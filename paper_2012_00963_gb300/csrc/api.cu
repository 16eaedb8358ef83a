// api.cu — the C ABI of libpdv (include/pdv.h): contexts, clouds and their
// device tables, single and batched spectrum requests (the batched launch is
// replayed from a captured CUDA graph), the launch-parameter autotuner, and
// the continuous-batching serving loop behind pdv_submit / pdv_poll.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pdv_internal.cuh"
#include "spectra.cuh"
#include "stepping.cuh"

using namespace pdv;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

// Select the context's device and drop any stale error state left in the
// runtime's per-thread "last error" by an earlier optional call.
static cudaError_t enter(int device) {
  cudaError_t e = cudaSetDevice(device);
  cudaGetLastError();
  return e;
}

static pdv_status fail(pdv_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? PDV_ENOMEM : PDV_ECUDA, "%s: %s", #x, \
                  cudaGetErrorString(e_));                                             \
  } while (0)

extern "C" const char* pdv_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ objects
struct Request;  // serving

constexpr unsigned long long kPoolKeep = 2ull << 30;   // bytes a context's pool keeps mapped

struct pdv_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  pdv_allocator alloc{};
  bool has_alloc = false;
  // the context's own stream-ordered pool: it keeps up to kPoolKeep bytes of
  // freed memory mapped across synchronisations, so per-call allocations do
  // not map fresh memory each time (the default pool releases at every sync)
  cudaMemPool_t pool = nullptr;
  int sm_count = 0;
  int max_smem = 0;                   // shared memory the transport's tables may use
  int smem_optin = 0;                 // the device's opt-in shared memory per block
  pdv_tuning tuning{};
  std::string tune_cache;              // pdv_autotune's JSON cache file (empty: none)
  std::string device_name;
  std::mutex mu;                      // serialises synchronous calls on the stream
  std::atomic<unsigned long long> launches{0};
  double last_transport_ms = 0.0;
  double last_model_ms = 0.0;
  unsigned long long last_steps = 0;
  unsigned long long last_events = 0;
  int last_grid = 0, last_block = 0;
  int last_fast = 0;      // 1: the last FP32 transport launch ran the common-configuration build
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // batched-graph cache
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    void* arena = nullptr;            // device arena of the batch (fixed pointers)
    size_t arena_bytes = 0;
    void* pinned = nullptr;           // pinned staging (set descriptors in, outputs out)
    size_t pinned_bytes = 0;
  };
  std::vector<GraphEntry> graphs;
  // serving
  std::thread worker;
  std::mutex smu;
  std::condition_variable scv;
  std::condition_variable done_cv;
  bool stop = false;
  std::map<pdv_ticket, std::shared_ptr<Request>> requests;
  std::deque<std::shared_ptr<Request>> active;
  pdv_ticket next_ticket = 1;
  cudaStream_t serve_stream = nullptr;
  int max_slots = 1024;                     // admitted requests not yet polled
  uint64_t mem_reserve = 256ull << 20;     // device memory admission keeps free
  unsigned long long quantum = 1ull << 21;   // packets per request per serving launch
  // pinned staging buffers for served outputs, reused by size class (page-
  // locking memory per request would cost milliseconds of latency)
  std::mutex pin_mu;
  std::map<size_t, std::vector<void*>> pinned_free;
  size_t mem_free = 0;
  std::chrono::steady_clock::time_point mem_checked{};
  // fixed-scratch entry point: the device address of the file-scope scratch
  // array on this context's device, and host buffers for the snapshot times,
  // all set up when the context is made (the call itself allocates nothing)
  char* static_scratch = nullptr;
  std::vector<double> static_ts;
  std::vector<int> static_idx;
  // debug build: the path trace armed by pdv_debug_set_trace for the next
  // synchronous spectrum call with per-packet records
  pdv_trace_vertex* trace_out = nullptr;
  int trace_n = 0, trace_max = 0;
};

static size_t pin_class(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  return c;
}

static void* pin_acquire(pdv_ctx* c, size_t bytes, size_t* cls) {
  *cls = pin_class(bytes);
  {
    std::lock_guard<std::mutex> lk(c->pin_mu);
    auto& v = c->pinned_free[*cls];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, *cls) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pin_release(pdv_ctx* c, void* p, size_t cls) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(c->pin_mu);
  c->pinned_free[cls].push_back(p);
}

struct pdv_cloud {
  pdv_ctx* ctx = nullptr;
  pdv_cloud_desc desc{};
  std::vector<double> prof_v, prof_f;
  double v_bot = 0, v_top = 0, d_s = 0, m0 = 0;
  double tau_tot = 0, q_ext = 0, albedo = 0, g_tab = 0;
  bool has_phase = false;
  CloudTables t;
  float* pn = nullptr;                // p(theta) / max p at the phase nodes (layer stepping)
  double max_dtheta = 0;              // largest spacing of the phase table's angles
  void* mass_arena = nullptr;
  void* phase_arena = nullptr;
};

// ------------------------------------------------------------------ memory
static void* ctx_alloc(pdv_ctx* c, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (c->has_alloc) return c->alloc.alloc(bytes, (void*)st, c->alloc.user);
  void* p = nullptr;
  const cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&p, bytes, c->pool, st)
                                : cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
static void ctx_free(pdv_ctx* c, void* p, cudaStream_t st) {
  if (!p) return;
  if (c->has_alloc) c->alloc.free(p, (void*)st, c->alloc.user);
  else cudaFreeAsync(p, st);
}

// Bump layout inside one allocation, 256-byte aligned pieces.
struct Layout {
  size_t bytes = 0;
  size_t add(size_t b) {
    const size_t o = bytes;
    bytes += (b + 255) & ~(size_t)255;
    return o;
  }
};

// ------------------------------------------------------------------ context
static cudaError_t static_scratch_lookup(char** out);

extern "C" pdv_status pdv_ctx_create(int device, void* cuda_stream, const pdv_allocator* alloc,
                                     pdv_ctx** out) {
  NvtxRange nvtx_range("pdv_ctx_create");
  if (!out) return fail(PDV_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(PDV_EINVAL, "device %d out of range", device);
  CK(enter(device));
  auto* c = new pdv_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(PDV_ECUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  if (alloc) {
    if (!alloc->alloc || !alloc->free) {
      if (c->own_stream) cudaStreamDestroy(c->stream);
      delete c;
      return fail(PDV_EINVAL, "allocator callbacks missing");
    }
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  if (!c->has_alloc) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
      unsigned long long keep = kPoolKeep;      // a cuuint64_t attribute
      cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      c->pool = nullptr;                 // fall back to the device's default pool
    }
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->device_name = prop.name;
    cudaGetLastError();
  }
  c->max_smem = transport_f32_max_smem();
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->tuning.block_threads = 256;
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  // Everything pdv_simulate_spectrum_static needs is made here, so that the
  // call itself allocates nothing: the scratch array's device address (which
  // loads this file's module and maps the array on this device), the
  // transport and normalisation kernels (loaded now, not at their first
  // launch, under the runtime's lazy module loading), and host buffers for
  // the snapshot times.
  cudaError_t e = static_scratch_lookup(&c->static_scratch);
  if (e == cudaSuccess) e = transport_preload();
  if (e != cudaSuccess) {
    pdv_ctx_destroy(c);
    return fail(PDV_ECUDA, "context set-up failed: %s", cudaGetErrorString(e));
  }
  c->static_ts.assign(3 * (size_t)kMaxSnap, 0.0);
  c->static_idx.assign((size_t)kMaxSnap, 0);
  *out = c;
  return PDV_OK;
}

static void serving_stop(pdv_ctx* c);

extern "C" pdv_status pdv_ctx_destroy(pdv_ctx* c) {
  NvtxRange nvtx_range("pdv_ctx_destroy");
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  enter(c->device);
  serving_stop(c);
  cudaStreamSynchronize(c->stream);
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.arena) ctx_free(c, g.arena, c->stream);
    if (g.pinned) cudaFreeHost(g.pinned);
  }
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->pinned_free)
    for (void* p : kv.second) cudaFreeHost(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  // released once its last allocation is freed (clouds are destroyed first)
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
  return PDV_OK;
}

extern "C" pdv_status pdv_get_stats(pdv_ctx* c, pdv_stats* out) {
  if (!c || !out) return fail(PDV_EINVAL, "NULL argument");
  out->kernel_launches = c->launches.load();
  out->last_transport_ms = c->last_transport_ms;
  out->last_events = c->last_events;
  out->transport_grid = c->last_grid;
  out->transport_block = c->last_block;
  out->last_model_ms = c->last_model_ms;
  out->last_steps = c->last_steps;
  out->transport_fast = c->last_fast;
  out->reserved = 0;
  return PDV_OK;
}

extern "C" pdv_status pdv_set_tuning(pdv_ctx* c, const pdv_tuning* t) {
  if (!c || !t) return fail(PDV_EINVAL, "NULL argument");
  if (t->block_threads && t->block_threads != 64 && t->block_threads != 128 &&
      t->block_threads != 256)
    return fail(PDV_EINVAL, "block_threads must be 64, 128 or 256");
  if (t->hist_mode < 0 || t->hist_mode > 2) return fail(PDV_EINVAL, "hist_mode must be 0..2");
  if (t->blocks_per_sm < 0) return fail(PDV_EINVAL, "negative blocks_per_sm");
  if (t->tile_packets && (t->tile_packets < 16 || t->tile_packets > 65536))
    return fail(PDV_EINVAL, "tile_packets must be 0 or in [16, 65536]");
  c->tuning = *t;
  if (!c->tuning.block_threads) c->tuning.block_threads = 256;
  return PDV_OK;
}

// ------------------------------------------------------------------ cloud
static pdv_status validate_cloud(const pdv_cloud_desc* d, double* v_bot, double* v_top) {
  if (!(d->rho_kg_m3 > 0)) return fail(PDV_EINVAL, "rho must be > 0");
  if (!(d->area_mass_mg_cm2 >= 0)) return fail(PDV_EINVAL, "area mass must be >= 0");
  if (!(d->d_median_um > 0)) return fail(PDV_EINVAL, "median diameter must be > 0");
  if (!(d->sigma_ln >= 0)) return fail(PDV_EINVAL, "sigma_ln must be >= 0");
  if (!(d->reflectivity >= 0 && d->reflectivity <= 1)) return fail(PDV_EINVAL, "reflectivity must be in [0,1]");
  if (d->surface_mode < 0 || d->surface_mode > 2) return fail(PDV_EINVAL, "bad surface_mode");
  if (!(d->v_fs > 0)) return fail(PDV_EINVAL, "v_fs must be > 0");
  if (d->table_nodes < 0 || d->table_nodes > kMaxTableNodes || (d->table_nodes && d->table_nodes < 16))
    return fail(PDV_EINVAL, "table_nodes must be 0 or in [16, %d]", kMaxTableNodes);
  if (d->profile_kind == PDV_PROFILE_EXPONENTIAL) {
    if (!(d->beta > 0)) return fail(PDV_EINVAL, "beta must be > 0");
    *v_bot = d->v_fs;
    *v_top = d->v_max > 0 ? d->v_max : d->v_fs * (1.0 + std::log(1.0e6) / d->beta);
    if (!(*v_top > *v_bot)) return fail(PDV_EINVAL, "v_max must exceed v_fs");
  } else if (d->profile_kind == PDV_PROFILE_TABULATED) {
    if (d->prof_n < 2 || d->prof_n > 65536 || !d->prof_v || !d->prof_dmdv)
      return fail(PDV_EINVAL, "tabulated profile needs 2..65536 points");
    for (int i = 0; i < d->prof_n; ++i) {
      if (!(d->prof_dmdv[i] > 0)) return fail(PDV_EINVAL, "dm/dv must be > 0");
      if (i && !(d->prof_v[i] > d->prof_v[i - 1])) return fail(PDV_EINVAL, "profile velocities must increase");
    }
    if (!(d->prof_v[0] >= d->v_fs)) return fail(PDV_EINVAL, "profile must start at or above v_fs");
    *v_bot = d->prof_v[0];
    *v_top = d->prof_v[d->prof_n - 1];
  } else {
    return fail(PDV_EINVAL, "bad profile_kind");
  }
  return PDV_OK;
}

static int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

extern "C" pdv_status pdv_create_cloud(pdv_ctx* c, const pdv_cloud_desc* d, pdv_cloud** out) {
  NvtxRange nvtx_range("pdv_create_cloud");
  if (!c || !d || !out) return fail(PDV_EINVAL, "NULL argument");
  *out = nullptr;
  double v_bot = 0, v_top = 0;
  pdv_status s = validate_cloud(d, &v_bot, &v_top);
  if (s != PDV_OK) return s;
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  auto* cl = new pdv_cloud();
  cl->ctx = c;
  cl->desc = *d;
  if (d->profile_kind == PDV_PROFILE_TABULATED) {
    cl->prof_v.assign(d->prof_v, d->prof_v + d->prof_n);
    cl->prof_f.assign(d->prof_dmdv, d->prof_dmdv + d->prof_n);
  }
  cl->desc.prof_v = nullptr;
  cl->desc.prof_dmdv = nullptr;
  cl->v_bot = v_bot;
  cl->v_top = v_top;
  cl->d_s = d->d_median_um * 1e-6 * std::exp(2.5 * d->sigma_ln * d->sigma_ln);
  cl->m0 = d->area_mass_mg_cm2 * 1e-2;
  const int n_v = d->table_nodes ? d->table_nodes : 2048;
  // two guide cells per node up to 4096 nodes (fewer search steps where the
  // mass fraction crowds near the top of the cloud), one above
  const int n_g = n_v <= 4096 ? 2 * next_pow2(n_v) : std::min(next_pow2(n_v), kMaxTableNodes);
  int lg = 0;
  while ((1 << lg) < n_g) ++lg;
  cl->t.n_v = n_v;
  cl->t.n_g = n_g;
  cl->t.g_shift = 62 - lg;
  const int pn = (int)cl->prof_v.size();
  Layout L;
  const size_t oSq = L.add(sizeof(unsigned long long) * (n_v + 1));
  const size_t oSd = L.add(sizeof(double) * (n_v + 1));
  const size_t ow = L.add(sizeof(float) * n_v);
  const size_t oG = L.add(sizeof(unsigned short) * (n_g + 1));
  const size_t opv = L.add(sizeof(double) * std::max(pn, 1));
  const size_t opf = L.add(sizeof(double) * std::max(pn, 1));
  const size_t opc = L.add(sizeof(double) * std::max(pn, 1));
  char* base = (char*)ctx_alloc(c, L.bytes, c->stream);
  if (!base) {
    delete cl;
    return fail(PDV_ENOMEM, "cloud table allocation failed");
  }
  cl->mass_arena = base;
  cl->t.Sq = (unsigned long long*)(base + oSq);
  cl->t.Sd = (double*)(base + oSd);
  cl->t.w = (float*)(base + ow);
  cl->t.G = (unsigned short*)(base + oG);
  double* dpv = (double*)(base + opv);
  double* dpf = (double*)(base + opf);
  double* dpc = (double*)(base + opc);
  cudaError_t e = cudaSuccess;
  if (pn) {
    e = cudaMemcpyAsync(dpv, cl->prof_v.data(), sizeof(double) * pn, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dpf, cl->prof_f.data(), sizeof(double) * pn, cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess)
    e = build_mass_table(d->profile_kind, d->beta, d->v_fs, v_bot, v_top, dpv, dpf, pn, dpc, n_v,
                         &cl->t, c->stream);
  c->launches += (d->profile_kind == PDV_PROFILE_TABULATED ? 4 : 3);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    ctx_free(c, base, c->stream);
    cudaStreamSynchronize(c->stream);
    delete cl;
    return fail(PDV_ECUDA, "mass table build failed: %s", cudaGetErrorString(e));
  }
  *out = cl;
  return PDV_OK;
}

extern "C" pdv_status pdv_set_phase_table(pdv_cloud* cl, int n, const double* theta,
                                          const double* p, double q_ext, double albedo) {
  NvtxRange nvtx_range("pdv_set_phase_table");
  if (!cl || !theta || !p) return fail(PDV_EINVAL, "NULL argument");
  if (n < 2 || n > kMaxPhase) return fail(PDV_EINVAL, "phase table needs 2..%d angles", kMaxPhase);
  if (std::fabs(theta[0]) > 1e-12 || std::fabs(theta[n - 1] - M_PI) > 1e-12)
    return fail(PDV_EINVAL, "theta must run from 0 to pi");
  double total = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(p[i] >= 0) || !std::isfinite(p[i])) return fail(PDV_EINVAL, "p must be finite and >= 0");
    if (i && !(theta[i] > theta[i - 1])) return fail(PDV_EINVAL, "theta must increase strictly");
    if (i) total += 0.5 * (p[i - 1] * std::sin(theta[i - 1]) + p[i] * std::sin(theta[i])) * (theta[i] - theta[i - 1]);
  }
  if (!(total > 0)) return fail(PDV_EINVAL, "phase function integrates to zero");
  bool uniform = true;
  for (int i = 0; i < n && uniform; ++i)
    uniform = std::fabs(theta[i] - M_PI * (double)i / (double)(n - 1)) <= 1e-12;
  if (!(q_ext >= 0) || !std::isfinite(q_ext)) return fail(PDV_EINVAL, "q_ext must be >= 0");
  if (!(albedo >= 0 && albedo <= 1)) return fail(PDV_EINVAL, "albedo must be in [0,1]");
  pdv_ctx* c = cl->ctx;
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  if (cl->phase_arena) {
    ctx_free(c, cl->phase_arena, c->stream);
    cl->phase_arena = nullptr;
    cl->has_phase = false;
  }
  const int ngp = (1 << kGuidePhaseLog) + 1;
  Layout L;
  const size_t oCq = L.add(sizeof(unsigned) * n);
  const size_t oth = L.add(sizeof(float) * n);
  const size_t odt = L.add(sizeof(float) * n);
  const size_t ocs = L.add(sizeof(float2) * n);
  const size_t ond = L.add(sizeof(uint2) * n);
  const size_t othd = L.add(sizeof(double) * n);
  const size_t oGp = L.add(sizeof(unsigned short) * ngp);
  const size_t oin = L.add(sizeof(double) * 2 * n);
  const size_t owk = L.add(sizeof(double) * 2 * n);
  const size_t og = L.add(sizeof(double));
  const size_t opn = L.add(sizeof(float) * n);
  char* base = (char*)ctx_alloc(c, L.bytes, c->stream);
  if (!base) return fail(PDV_ENOMEM, "phase table allocation failed");
  // p / max p for the layer-stepping scheme's acceptance-rejection
  double p_max = 0.0;
  for (int i = 0; i < n; ++i) p_max = std::max(p_max, p[i]);
  std::vector<float> pn(n);
  for (int i = 0; i < n; ++i) pn[i] = (float)(p[i] / p_max);
  cl->pn = (float*)(base + opn);
  cl->phase_arena = base;
  cl->t.Cq = (unsigned*)(base + oCq);
  cl->t.thpi = (float*)(base + oth);
  cl->t.dthpi = (float*)(base + odt);
  cl->t.cs = (float2*)(base + ocs);
  cl->t.node = (uint2*)(base + ond);
  cl->t.th_d = (double*)(base + othd);
  cl->t.Gp = (unsigned short*)(base + oGp);
  cl->t.n_p = n;
  cl->t.phase_uniform = uniform ? 1 : 0;
  double* din = (double*)(base + oin);
  double* dwk = (double*)(base + owk);
  double* dg = (double*)(base + og);
  cudaError_t e = cudaMemcpyAsync(din, theta, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(din + n, p, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cl->pn, pn.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream);
  // (cos theta_i, sin theta_i) of the nodes: the FP32 walk's angle tables
  std::vector<float2> cs(n);
  cl->max_dtheta = 0;
  for (int i = 0; i < n; ++i) {
    cs[i] = make_float2((float)std::cos(theta[i]), (float)std::sin(theta[i]));
    if (i) cl->max_dtheta = std::max(cl->max_dtheta, theta[i] - theta[i - 1]);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cl->t.cs, cs.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = build_phase_cdf(din, din + n, n, dwk, &cl->t, dg, c->stream);
  c->launches += 6;
  double g = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&g, dg, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(PDV_ECUDA, "phase table build failed: %s", cudaGetErrorString(e));
  cl->g_tab = g;
  cl->q_ext = q_ext;
  cl->albedo = albedo;
  // Eq. 10 with the Sauter mean of the number log-normal (Eq. 21, d_s = <d^3>/<d^2>)
  cl->tau_tot = 3.0 * cl->m0 * q_ext / (2.0 * cl->desc.rho_kg_m3 * cl->d_s);
  cl->has_phase = true;
  return PDV_OK;
}

extern "C" pdv_status pdv_cloud_get_info(const pdv_cloud* cl, pdv_cloud_info* out) {
  if (!cl || !out) return fail(PDV_EINVAL, "NULL argument");
  out->tau_tot = cl->tau_tot;
  out->v_bot = cl->v_bot;
  out->v_top = cl->v_top;
  out->d_sauter_um = cl->d_s * 1e6;
  out->g_table = cl->g_tab;
  out->q_ext = cl->q_ext;
  out->albedo = cl->albedo;
  out->table_nodes = cl->t.n_v;
  out->has_phase = cl->has_phase ? 1 : 0;
  return PDV_OK;
}

extern "C" pdv_status pdv_destroy_cloud(pdv_cloud* cl) {
  if (!cl) return fail(PDV_EINVAL, "cloud is NULL");
  pdv_ctx* c = cl->ctx;
  enter(c->device);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStreamSynchronize(c->stream);
    if (c->serve_stream) cudaStreamSynchronize(c->serve_stream);
    ctx_free(c, cl->mass_arena, c->stream);
    ctx_free(c, cl->phase_arena, c->stream);
    cudaStreamSynchronize(c->stream);
  }
  delete cl;
  return PDV_OK;
}

extern "C" pdv_status pdv_phase_hg(double g, int n, double* theta, double* p) {
  if (!theta || !p || n < 2) return fail(PDV_EINVAL, "need n >= 2 and output arrays");
  if (!(g > -1 && g < 1)) return fail(PDV_EINVAL, "g must be in (-1, 1)");
  for (int j = 0; j < n; ++j) {
    theta[j] = M_PI * (double)j / (double)(n - 1);
    const double den = 1.0 + g * g - 2.0 * g * std::cos(theta[j]);
    p[j] = (1.0 - g * g) / (4.0 * M_PI * den * std::sqrt(den));
  }
  return PDV_OK;
}

struct AllocCb {
  pdv_ctx* c;
  cudaStream_t st;
};
static void* mie_alloc(size_t b, void* u) {
  auto* a = (AllocCb*)u;
  return ctx_alloc(a->c, b, a->st);
}
static void mie_free(void* p, void* u) {
  auto* a = (AllocCb*)u;
  ctx_free(a->c, p, a->st);
}

extern "C" pdv_status pdv_mie_table(pdv_ctx* c, double m_re, double m_im, double wavelength_nm,
                                    double d_median_um, double sigma_ln, int n_size, int n_angle,
                                    double* theta, double* p, double* q_ext, double* albedo,
                                    double* g) {
  NvtxRange nvtx_range("pdv_mie_table");
  if (!c || !theta || !p) return fail(PDV_EINVAL, "NULL argument");
  if (!(m_re > 0) || !(m_im >= 0)) return fail(PDV_EINVAL, "need Re m > 0 and Im m >= 0");
  if (!(wavelength_nm > 0) || !(d_median_um > 0) || !(sigma_ln >= 0) || sigma_ln > 3)
    return fail(PDV_EINVAL, "bad size distribution or wavelength");
  if (n_angle < 2 || n_angle > kMaxPhase) return fail(PDV_EINVAL, "n_angle out of range");
  if (sigma_ln > 0 && (n_size < 2 || n_size > 4096)) return fail(PDV_EINVAL, "n_size must be in [2, 4096]");
  const double lam = wavelength_nm * 1e-9, dm = d_median_um * 1e-6;
  const double x_hi = M_PI * dm * std::exp(6.0 * sigma_ln) / lam;
  if (x_hi > 20000.0) return fail(PDV_EINVAL, "size parameter %.0f above 20000", x_hi);
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  Layout L;
  const size_t ot = L.add(sizeof(double) * n_angle);
  const size_t op = L.add(sizeof(double) * n_angle);
  const size_t oq = L.add(sizeof(double) * 3);
  char* base = (char*)ctx_alloc(c, L.bytes, c->stream);
  if (!base) return fail(PDV_ENOMEM, "Mie output allocation failed");
  AllocCb cb{c, c->stream};
  cudaError_t e = mie_table_device(m_re, m_im, lam, dm, sigma_ln, n_size, n_angle,
                                   (double*)(base + ot), (double*)(base + op), (double*)(base + oq),
                                   c->stream, mie_alloc, mie_free, &cb);
  c->launches += 5;
  double q3[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(theta, base + ot, sizeof(double) * n_angle, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, base + op, sizeof(double) * n_angle, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q3, base + oq, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  ctx_free(c, base, c->stream);
  cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? PDV_ENOMEM : PDV_ECUDA,
                                    "Mie table failed: %s", cudaGetErrorString(e));
  if (q_ext) *q_ext = q3[0];
  if (albedo) *albedo = q3[1];
  if (g) *g = q3[2];
  return PDV_OK;
}

// ------------------------------------------------------------------ requests
static pdv_status validate_request(const pdv_request* r) {
  if (!r) return fail(PDV_EINVAL, "request is NULL");
  if (!r->cloud) return fail(PDV_EINVAL, "request has no cloud");
  if (!r->cloud->has_phase) return fail(PDV_EINVAL, "cloud has no phase table");
  if (r->n_snap < 1 || r->n_snap > kMaxSnap || !r->t_snap_us) return fail(PDV_EINVAL, "n_snap must be in [1, %d]", kMaxSnap);
  if (r->n_bins < 1 || r->n_bins > kMaxBins) return fail(PDV_EINVAL, "n_bins must be in [1, %d]", kMaxBins);
  if (!(r->v_hi > r->v_lo)) return fail(PDV_EINVAL, "v_hi must exceed v_lo");
  if (r->n_packets < 1 || r->n_packets > 4000000000ull) return fail(PDV_EINVAL, "n_packets must be in [1, 4e9]");
  if (r->packet_begin > ~0ull - r->n_packets) return fail(PDV_EINVAL, "packet range overflows");
  if (r->precision != PDV_PREC_FP32 && r->precision != PDV_PREC_FP64) return fail(PDV_EINVAL, "bad precision");
  if (!r->out_spectrum) return fail(PDV_EINVAL, "out_spectrum is required");
  if (r->out_packets && r->n_packets > ((r->flags & PDV_OUT_DEVICE) ? (1ull << 28) : (1ull << 26)))
    return fail(PDV_EINVAL, "packet dumps need n_packets <= 2^26 (2^28 into device memory)");
  if (r->flags & ~(PDV_OUT_DEVICE | PDV_PER_DV | PDV_IMPLICIT_CAPTURE | PDV_TEST_HORIZONTAL_LAUNCH |
                   PDV_TEST_DEBUG_CHECK))
    return fail(PDV_EINVAL, "unknown flags");
  if ((r->flags & PDV_TEST_DEBUG_CHECK) && !kDebugBuild)
    return fail(PDV_EINVAL, "PDV_TEST_DEBUG_CHECK needs the debug build (libpdv_debug.so)");
  if (r->n_layers && (r->flags & PDV_TEST_HORIZONTAL_LAUNCH))
    return fail(PDV_EINVAL, "the horizontal launch runs with exact free paths only (n_layers = 0)");
  if (r->reserved) return fail(PDV_EINVAL, "reserved must be 0");
  if (r->n_layers && r->precision != PDV_PREC_FP32)
    return fail(PDV_EINVAL, "the layer-stepping scheme runs in FP32");
  if (r->n_layers && (r->flags & PDV_IMPLICIT_CAPTURE))
    return fail(PDV_EINVAL, "implicit capture runs with exact free paths only (n_layers = 0)");
  const pdv_probe& pr = r->probe;
  if (!(pr.z_probe_mm > 0) || !(pr.beam_radius_mm >= 0) || !std::isfinite(pr.aperture_radius_mm) ||
      !(pr.cone_half_angle_rad > 0))
    return fail(PDV_EINVAL, "bad probe geometry");
  for (int s = 0; s < r->n_snap; ++s) {
    const double t = r->t_snap_us[s];
    if (!(t > 0) || !std::isfinite(t)) return fail(PDV_EINVAL, "snapshot times must be > 0");
    if (!(r->cloud->v_top * t * 1e-6 < pr.z_probe_mm * 1e-3))
      return fail(PDV_EINVAL, "top of the cloud at t = %g us reaches the probe plane", t);
  }
  return PDV_OK;
}

static SetDesc make_set(const pdv_request* r) {
  const pdv_cloud* cl = r->cloud;
  SetDesc d;
  memset(&d, 0, sizeof d);
  d.Sq = cl->t.Sq; d.Sd = cl->t.Sd; d.w = cl->t.w; d.G = cl->t.G;
  d.Cq = cl->t.Cq; d.thpi = cl->t.thpi; d.dthpi = cl->t.dthpi; d.th_d = cl->t.th_d; d.Gp = cl->t.Gp;
  d.cs = cl->t.cs;
  d.node = cl->t.node;
  d.n_v = cl->t.n_v; d.n_g = cl->t.n_g; d.g_shift = cl->t.g_shift; d.n_p = cl->t.n_p;
  d.phase_uniform = cl->t.phase_uniform;
  d.inv_nm1 = (float)(1.0 / (double)(cl->t.n_p - 1));
  d.angle_table = cl->max_dtheta <= 3.1e-3 ? 1 : 0;
  d.n_snap = r->n_snap; d.n_bins = r->n_bins;
  d.surface_mode = cl->desc.surface_mode;
  d.cone_all = r->probe.cone_half_angle_rad >= 0.5 * M_PI;
  d.ap_all = !(r->probe.aperture_radius_mm > 0);
  d.omega_q = (unsigned)std::floor(cl->albedo * 16777216.0 + 0.5);
  d.stream_id = r->stream_id;
  d.max_events = r->max_events ? std::min(r->max_events, 0xfffffffeu) : 1000000u;
  d.implicit = (r->flags & PDV_IMPLICIT_CAPTURE) ? 1u : 0u;
  d.launch_horizontal = (r->flags & PDV_TEST_HORIZONTAL_LAUNCH) ? 1 : 0;
  d.debug_check = (r->flags & PDV_TEST_DEBUG_CHECK) ? 1 : 0;
  d.t_trace = r->t_snap_us[0] * 1e-6;
  d.absorb_gate = d.implicit ? 0u : d.omega_q;
  d.R_q = (unsigned long long)std::floor(cl->desc.reflectivity * kTwo32 + 0.5);
  d.seed = r->seed;
  d.packet_begin = r->packet_begin;
  d.n_packets = r->n_packets;
  d.norm_packets = r->n_packets;
  d.tau_tot = cl->tau_tot;
  d.inv_tau = 1.0 / cl->tau_tot;   // +inf for an empty cloud: every flight leaves it
  d.v_bot = cl->v_bot;
  d.dv = (cl->v_top - cl->v_bot) / cl->t.n_v;
  d.v_top = cl->v_top;
  d.v_fs = cl->desc.v_fs;
  d.z_probe = r->probe.z_probe_mm * 1e-3;
  d.r_beam = r->probe.beam_radius_mm * 1e-3;
  const double rap = r->probe.aperture_radius_mm * 1e-3;
  d.r_ap2 = rap * rap;
  d.cos_alpha = std::cos(r->probe.cone_half_angle_rad);
  d.v_lo = r->v_lo;
  d.inv_dbin = (double)r->n_bins / (r->v_hi - r->v_lo);
  d.inv_tau_f = (float)d.inv_tau;
  d.v_bot_f = (float)d.v_bot; d.dv_f = (float)d.dv; d.v_top_f = (float)d.v_top; d.v_fs_f = (float)d.v_fs;
  d.z_probe_f = (float)d.z_probe; d.r_beam_f = (float)d.r_beam; d.r_ap2_f = (float)d.r_ap2;
  d.cos_alpha_f = (float)d.cos_alpha; d.v_lo_f = (float)d.v_lo; d.inv_dbin_f = (float)d.inv_dbin;
  d.expo = cl->desc.profile_kind == PDV_PROFILE_EXPONENTIAL ? 1 : 0;
  if (d.expo) {
    // Eq. 20 cut at v_top and renormalised: S(v) = (1 - exp(-beta (v/v_fs - 1))) / E, so
    // 1 - S E = (1 - S) + S eps with eps = 1 - E, and v = v_fs (1 - ln(1 - S E) / beta)
    const double x = cl->desc.beta * (cl->v_top / cl->desc.v_fs - 1.0);
    d.eps_f = (float)std::exp(-x);
    d.eps30_f = std::ldexp(d.eps_f, -30);
    d.lg_c_f = (float)(cl->desc.v_fs * M_LN2 / cl->desc.beta);
    d.dvds_c_f = (float)(cl->desc.v_fs * -std::expm1(-x) / cl->desc.beta);
    d.vb_d = cl->desc.v_fs / cl->desc.beta;
    d.E_d = -std::expm1(-x);
  }
  // Philox round keys: the key after i Weyl increments (Salmon et al.), mod 2^32
  for (unsigned i = 0; i < 10; ++i) {
    d.rk[i].x = (unsigned)((uint32_t)r->seed + i * 0x9E3779B9u);
    d.rk[i].y = (unsigned)((uint32_t)(r->seed >> 32) + i * 0xBB67AE85u);
  }
  return d;
}

// Snapshot times as the kernels read them: the times in request order
// (seconds), the same times ascending, and the request index of each
// ascending time (as a double). The FP32 kernel walks the ascending list to
// visit only the times at which an escaping packet is inside the aperture.
static size_t time_words(int n_snap) { return 3 * (size_t)n_snap; }

static void fill_times_into(const pdv_request* r, double* out, int* idx) {
  const int n = r->n_snap;
  for (int i = 0; i < n; ++i) idx[i] = i;
  const double* t = r->t_snap_us;
  std::sort(idx, idx + n, [t](int a, int b) { return t[a] < t[b] || (t[a] == t[b] && a < b); });
  for (int i = 0; i < n; ++i) {
    out[i] = t[i] * 1e-6;
    out[n + i] = t[idx[i]] * 1e-6;
    out[2 * n + i] = (double)idx[i];
  }
}

static void fill_times(const pdv_request* r, double* out) {
  int idx[kMaxSnap];
  fill_times_into(r, out, idx);
}

// Device buffers of one request: set descriptor, counters, histogram,
// snapshot times and staged outputs.
struct ReqBuffers {
  size_t o_set, o_ctr, o_cnt, o_hist, o_t, o_spec, o_craw, o_cout, o_pk, o_ptr_spec, o_ptr_cnt,
      o_ptr_raw, o_flags, o_steps;
  size_t bytes;
};

static ReqBuffers plan_request(const pdv_request* r, bool device_out) {
  ReqBuffers b;
  Layout L;
  const size_t row = hist_row(r->n_bins);
  b.o_set = L.add(sizeof(SetDesc));
  b.o_ctr = L.add(sizeof(unsigned long long));
  b.o_cnt = L.add(sizeof(unsigned long long) * C_NCOUNT);
  b.o_hist = L.add(sizeof(unsigned long long) * row * r->n_snap);
  b.o_t = L.add(sizeof(double) * time_words(r->n_snap));
  b.o_spec = device_out ? 0 : L.add(sizeof(double) * (size_t)r->n_snap * r->n_bins);
  b.o_craw = (!device_out && r->out_raw) ? L.add(sizeof(unsigned long long) * (size_t)r->n_snap * (r->n_bins + 2)) : 0;
  b.o_cout = (!device_out && r->out_counters) ? L.add(sizeof(pdv_counters) * r->n_snap) : 0;
  b.o_pk = (!device_out && r->out_packets) ? L.add(sizeof(pdv_packet_record) * r->n_packets) : 0;
  b.o_ptr_spec = L.add(sizeof(void*));
  b.o_ptr_cnt = L.add(sizeof(void*));
  b.o_ptr_raw = L.add(sizeof(void*));
  b.o_flags = L.add(sizeof(unsigned));
  b.o_steps = L.add(sizeof(unsigned long long));
  b.bytes = L.bytes;
  return b;
}

static size_t set_smem(const SetDesc& d, int hm) {
  return transport_f32_smem(d.n_v, d.n_g, d.n_p, d.n_snap, d.n_bins, hm, d.phase_uniform, d.ap_all,
                            d.expo, d.angle_table);
}

static int pick_hist_mode(const pdv_ctx* c, const SetDesc& d) {
  if (c->tuning.hist_mode == 1) return 1;
  const size_t tables = set_smem(d, 1);
  const size_t priv = set_smem(d, 2);
  if (c->tuning.hist_mode == 2) return priv <= (size_t)c->max_smem ? 2 : 1;
  // auto: privatise when the histogram is small next to the tables
  return (priv - tables) <= 16384 && priv <= (size_t)c->max_smem ? 2 : 1;
}

// Launch geometry of the persistent FP32 kernel for given shared memory.
static pdv_status f32_geometry(pdv_ctx* c, size_t smem, int hist_mode, bool dump, bool impl,
                               bool fast, int* grid, int* block, bool one = false) {
  const int bt = c->tuning.block_threads ? c->tuning.block_threads : 256;
  int occ = 0;
  CK(transport_f32_occupancy(bt, smem, hist_mode, dump, impl, one, fast, &occ));
  if (occ < 1) return fail(PDV_EINVAL, "tables need %zu bytes of shared memory, too many for one block", smem);
  int bps = c->tuning.blocks_per_sm ? std::min(c->tuning.blocks_per_sm, occ) : occ;
  *grid = c->sm_count * bps;
  *block = bt;
  return PDV_OK;
}

// Debug build: after a synchronous call's kernels have finished, a failed
// index check (left in the device words until pdv_debug_get resets them)
// turns the call's status into PDV_EDEBUG. The release build has no checks.
static pdv_status debug_after(pdv_ctx* c) {
  if (!kDebugBuild) return PDV_OK;
  DebugWord a{}, b{};
  CK(transport_debug_io(&a, false, c->stream));
  CK(stepping_debug_io(&b, false, c->stream));
  const DebugWord& f = a.violations ? a : b;
  if (!f.violations) return PDV_OK;
  return fail(PDV_EDEBUG, "index check failed: site %u, index %lld, bound %lld (%llu failed checks)",
              f.site, (long long)f.index, (long long)f.bound,
              (unsigned long long)(a.violations + b.violations));
}

// Enqueue the transport of one request whose buffers are at `base`
// (descriptor already uploaded). Returns the number of kernels launched.
static pdv_status enqueue_transport(pdv_ctx* c, const pdv_request* r, const SetDesc& d,
                                    char* base, const ReqBuffers& b, cudaStream_t st,
                                    bool timed) {
  if (r->n_layers) {
    // the paper's layer stepping (Section II.B steps (2)-(6))
    const pdv_cloud* cl = r->cloud;
    const double span = cl->v_top - cl->v_bot;
    const double h_v = (cl->v_top - cl->desc.v_fs) / (double)r->n_layers;
    StepConst sc;
    sc.P_fs = std::llround((cl->desc.v_fs - cl->v_bot) / span * kTwo62);
    sc.h_P = std::llround(h_v / span * kTwo62);
    sc.h_v = (float)h_v;
    sc.v_per_P = (float)(span / kTwo62);
    sc.tau_S = (float)(cl->tau_tot / kTwo62);
    sc.tau_hv_dv = (float)(cl->tau_tot / kTwo62 * h_v / (span / cl->t.n_v));
    sc.key2x = (unsigned)r->seed ^ 0xA4093822u;
    sc.key2y = (unsigned)(r->seed >> 32) ^ r->stream_id;
    sc.eps_P = std::llround(1e-6 * (kTwo62 - (double)sc.P_fs));
    sc.expo = cl->desc.profile_kind == PDV_PROFILE_EXPONENTIAL ? 1 : 0;
    sc.b_vfs = (float)(cl->desc.beta / cl->desc.v_fs);
    sc.invE = sc.expo ? (float)(1.0 / -std::expm1(-cl->desc.beta * (cl->v_top / cl->desc.v_fs - 1.0))) : 0.f;
    sc.tau_f = (float)cl->tau_tot;
    sc.shift_d = 0;
    while ((sc.h_P >> sc.shift_d) >= (1ll << 30)) ++sc.shift_d;
    sc.ff = sc.h_P <= (1ll << 56) ? 1 : 0;
    if (sc.P_fs < -(1ll << 62))
      return fail(PDV_EINVAL, "layer stepping needs the cloud to start within one cloud height of the free surface");
    const size_t smem = transport_step_smem(d.n_v, d.n_p, d.n_snap, d.phase_uniform);
    if (smem > (size_t)c->max_smem) return fail(PDV_EINVAL, "tables need %zu bytes of shared memory", smem);
    int occ = 0;
    CK(transport_step_occupancy(smem, &occ));
    if (occ < 1) return fail(PDV_EINVAL, "layer-stepping kernel does not fit");
    const unsigned long long want = (r->n_packets + 255) / 256;
    const int grid = (int)std::min<unsigned long long>(want, (unsigned long long)c->sm_count * occ);
    CK(cudaMemsetAsync(base + b.o_steps, 0, sizeof(unsigned long long), st));
    if (timed) cudaEventRecord(c->ev0, st);
    CK(launch_transport_step((const SetDesc*)(base + b.o_set), cl->pn, sc,
                             (unsigned long long*)(base + b.o_ctr),
                             (unsigned long long*)(base + b.o_steps), std::max(grid, 1), smem, st));
    if (timed) cudaEventRecord(c->ev1, st);
    c->last_grid = std::max(grid, 1);
    c->last_block = 256;
    c->last_fast = 0;
    c->launches += 1;
    return PDV_OK;
  }
  if (timed) cudaEventRecord(c->ev0, st);
  if (r->precision == PDV_PREC_FP32) {
    const int hm = pick_hist_mode(c, d);
    const bool dump = d.packets != nullptr;
    const size_t smem = set_smem(d, hm);
    if (smem > (size_t)c->max_smem) return fail(PDV_EINVAL, "tables need %zu bytes of shared memory (max %d)", smem, c->max_smem);
    int grid = 0, block = 0;
    const bool impl = d.implicit != 0;
    const bool fast = transport_fast_set(d);
    pdv_status s = f32_geometry(c, smem, hm, dump, impl, fast, &grid, &block, true);
    if (s != PDV_OK) return s;
    launch_transport_f32_one(d, (unsigned long long*)(base + b.o_ctr), grid, block, smem, hm, dump,
                             impl, fast, (unsigned)c->tuning.tile_packets, st);
    c->last_grid = grid;
    c->last_block = block;
    c->last_fast = fast && !dump;
  } else {
    const unsigned long long want = (r->n_packets + 255) / 256;
    const int grid = (int)std::min<unsigned long long>(want, (unsigned long long)c->sm_count * 8);
    launch_transport_f64((const SetDesc*)(base + b.o_set), std::max(grid, 1), 256, st);
    c->last_grid = std::max(grid, 1);
    c->last_block = 256;
    c->last_fast = 0;
  }
  c->launches += 1;
  CK(cudaGetLastError());
  if (timed) cudaEventRecord(c->ev1, st);
  return PDV_OK;
}

extern "C" pdv_status pdv_simulate_spectrum(pdv_ctx* c, const pdv_request* r) {
  NvtxRange nvtx_range("pdv_simulate_spectrum");
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  pdv_status s = validate_request(r);
  if (s != PDV_OK) return s;
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  const bool dev_out = (r->flags & PDV_OUT_DEVICE) != 0;
  const ReqBuffers b = plan_request(r, dev_out);
  cudaStream_t st = c->stream;
  char* base = (char*)ctx_alloc(c, b.bytes, st);
  if (!base) return fail(PDV_ENOMEM, "request allocation of %zu bytes failed", b.bytes);
  struct Guard {
    pdv_ctx* c; char* p; cudaStream_t st;
    ~Guard() { ctx_free(c, p, st); cudaStreamSynchronize(st); }
  } guard{c, base, st};

  SetDesc d = make_set(r);
  d.t_snap = (const double*)(base + b.o_t);
  d.hist = (unsigned long long*)(base + b.o_hist);
  d.cnt = (unsigned long long*)(base + b.o_cnt);
  d.packets = r->out_packets ? (dev_out ? r->out_packets : (pdv_packet_record*)(base + b.o_pk)) : nullptr;
  // debug build: the armed path trace of the first packets
  struct TraceGuard {
    pdv_ctx* c; void* p; cudaStream_t st;
    ~TraceGuard() { if (p) ctx_free(c, p, st); }
  } tguard{c, nullptr, st};
  int n_tr = 0;
  if (c->trace_n > 0 && r->out_packets && !r->n_layers) {
    n_tr = (int)std::min<uint64_t>((uint64_t)c->trace_n, r->n_packets);
    const size_t tb = sizeof(pdv_trace_vertex) * (size_t)n_tr * (size_t)c->trace_max;
    tguard.p = ctx_alloc(c, tb, st);
    if (!tguard.p) return fail(PDV_ENOMEM, "path trace allocation of %zu bytes failed", tb);
    CK(cudaMemsetAsync(tguard.p, 0xFF, tb, st));            // kind -1 in every unused slot
    d.trace = (pdv_trace_vertex*)tguard.p;
    d.n_trace = n_tr;
    d.max_vtx = c->trace_max;
  }
  std::vector<double> ts(time_words(r->n_snap));
  fill_times(r, ts.data());
  double* spec = dev_out ? r->out_spectrum : (double*)(base + b.o_spec);
  pdv_counters* cout = r->out_counters ? (dev_out ? r->out_counters : (pdv_counters*)(base + b.o_cout)) : nullptr;
  unsigned long long* raw = r->out_raw ? (dev_out ? (unsigned long long*)r->out_raw : (unsigned long long*)(base + b.o_craw)) : nullptr;
  const unsigned flags = r->flags;
  CK(cudaMemcpyAsync(base + b.o_t, ts.data(), sizeof(double) * ts.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + b.o_set, &d, sizeof d, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + b.o_ptr_spec, &spec, sizeof spec, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + b.o_ptr_cnt, &cout, sizeof cout, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + b.o_ptr_raw, &raw, sizeof raw, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + b.o_flags, &flags, sizeof flags, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(base + b.o_ctr, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(base + b.o_cnt, 0, sizeof(unsigned long long) * C_NCOUNT, st));
  CK(cudaMemsetAsync(base + b.o_hist, 0, sizeof(unsigned long long) * hist_row(r->n_bins) * r->n_snap, st));
  {
    NvtxRange nvtx_launch("pdv transport launch");
    s = enqueue_transport(c, r, d, base, b, st, true);
    if (s != PDV_OK) return s;
  }
  {
    NvtxRange nvtx_norm("pdv normalise");
    launch_normalise((const SetDesc*)(base + b.o_set), 1, (double* const*)(base + b.o_ptr_spec),
                     (pdv_counters* const*)(base + b.o_ptr_cnt),
                     (unsigned long long* const*)(base + b.o_ptr_raw),
                     (const unsigned*)(base + b.o_flags), r->n_snap, st);
  }
  c->launches += 1;
  CK(cudaGetLastError());
  if (!dev_out) {
    CK(cudaMemcpyAsync(r->out_spectrum, spec, sizeof(double) * (size_t)r->n_snap * r->n_bins, cudaMemcpyDeviceToHost, st));
    if (r->out_counters) CK(cudaMemcpyAsync(r->out_counters, cout, sizeof(pdv_counters) * r->n_snap, cudaMemcpyDeviceToHost, st));
    if (r->out_raw) CK(cudaMemcpyAsync(r->out_raw, raw, sizeof(unsigned long long) * (size_t)r->n_snap * (r->n_bins + 2), cudaMemcpyDeviceToHost, st));
    if (r->out_packets) CK(cudaMemcpyAsync(r->out_packets, d.packets, sizeof(pdv_packet_record) * r->n_packets, cudaMemcpyDeviceToHost, st));
  }
  unsigned long long ev = 0, steps = 0;
  CK(cudaMemcpyAsync(&ev, base + b.o_cnt + sizeof(unsigned long long) * C_EVENTS, sizeof ev, cudaMemcpyDeviceToHost, st));
  if (r->n_layers)
    CK(cudaMemcpyAsync(&steps, base + b.o_steps, sizeof steps, cudaMemcpyDeviceToHost, st));
  if (n_tr) {
    const size_t row_b = sizeof(pdv_trace_vertex) * (size_t)c->trace_max;
    CK(cudaMemcpyAsync(c->trace_out, tguard.p, row_b * n_tr, cudaMemcpyDeviceToHost, st));
    if (n_tr < c->trace_n) memset((char*)c->trace_out + row_b * n_tr, 0xFF, row_b * (c->trace_n - n_tr));
  }
  CK(cudaStreamSynchronize(st));
  if (n_tr) {
    c->trace_n = 0;                               // one call per arming
    c->trace_out = nullptr;
  }
  c->last_steps = steps;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->last_transport_ms = ms;
  cudaGetLastError();
  c->last_events = ev;
  return debug_after(c);
}

// ------------------------------------------------------------------ batches
// All FP32 requests of a batch run in one persistent launch: the kernel walks
// the set list, so blocks move to the next set with packets left. The device
// work (counter/histogram clears, transport, normalisation) is captured once
// per batch shape into a CUDA graph whose device arena stays fixed, and
// replayed; per-call data (set descriptors, output pointers) is uploaded into
// that arena before each replay.
struct BatchLayout {
  size_t o_sets, o_ctr, o_cnt, o_hist, o_t, o_pspec, o_pcnt, o_praw, o_flags, bytes;
  std::vector<size_t> o_hist_i, o_t_i, o_spec_i, o_raw_i, o_cout_i, o_pk_i;
  size_t hist_words = 0;
};

static BatchLayout plan_batch(const pdv_request* rs, int n) {
  BatchLayout B;
  Layout L;
  B.o_sets = L.add(sizeof(SetDesc) * n);
  B.o_ctr = L.add(sizeof(unsigned long long) * n);
  B.o_cnt = L.add(sizeof(unsigned long long) * C_NCOUNT * n);
  size_t hw = 0;
  for (int i = 0; i < n; ++i) hw += (size_t)hist_row(rs[i].n_bins) * rs[i].n_snap;
  B.hist_words = hw;
  B.o_hist = L.add(sizeof(unsigned long long) * hw);
  size_t tw = 0;
  for (int i = 0; i < n; ++i) tw += time_words(rs[i].n_snap);
  B.o_t = L.add(sizeof(double) * tw);
  B.o_pspec = L.add(sizeof(void*) * n);
  B.o_pcnt = L.add(sizeof(void*) * n);
  B.o_praw = L.add(sizeof(void*) * n);
  B.o_flags = L.add(sizeof(unsigned) * n);
  size_t h = 0, t = 0;
  for (int i = 0; i < n; ++i) {
    const pdv_request& r = rs[i];
    const bool dev = (r.flags & PDV_OUT_DEVICE) != 0;
    B.o_hist_i.push_back(B.o_hist + sizeof(unsigned long long) * h);
    B.o_t_i.push_back(B.o_t + sizeof(double) * t);
    h += (size_t)hist_row(r.n_bins) * r.n_snap;
    t += time_words(r.n_snap);
    B.o_spec_i.push_back(dev ? 0 : L.add(sizeof(double) * (size_t)r.n_snap * r.n_bins));
    B.o_raw_i.push_back((!dev && r.out_raw) ? L.add(sizeof(unsigned long long) * (size_t)r.n_snap * (r.n_bins + 2)) : 0);
    B.o_cout_i.push_back((!dev && r.out_counters) ? L.add(sizeof(pdv_counters) * r.n_snap) : 0);
    B.o_pk_i.push_back((!dev && r.out_packets) ? L.add(sizeof(pdv_packet_record) * r.n_packets) : 0);
  }
  B.bytes = L.bytes;
  return B;
}

static std::string batch_key(const pdv_ctx* c, const pdv_request* rs, int n, int grid, int block,
                             size_t smem, int hm, bool dump) {
  std::string k;
  char buf[128];
  snprintf(buf, sizeof buf, "%d|%d|%d|%zu|%d|%d|%d|", n, grid, block, smem, hm, (int)dump,
           c->tuning.tile_packets);
  k += buf;
  for (int i = 0; i < n; ++i) {
    const pdv_request& r = rs[i];
    snprintf(buf, sizeof buf, "%d,%d,%u,%d,%d,%d,%llu;", r.n_snap, r.n_bins, r.flags,
             r.out_raw != nullptr, r.out_counters != nullptr, r.out_packets != nullptr,
             r.out_packets ? (unsigned long long)r.n_packets : 0ull);
    k += buf;
  }
  return k;
}

static pdv_status run_batch_f32(pdv_ctx* c, const pdv_request* rs, int n, bool timed,
                                float* transport_ms) {
  cudaStream_t st = c->stream;
  // launch geometry for the largest staged tables of the batch
  std::vector<SetDesc> sets(n);
  size_t smem = 0;
  int hm = 2;
  bool dump = false, impl = false, fast = true;
  for (int i = 0; i < n; ++i) {
    sets[i] = make_set(&rs[i]);
    if (pick_hist_mode(c, sets[i]) == 1) hm = 1;
    dump = dump || rs[i].out_packets != nullptr;
    impl = impl || sets[i].implicit != 0;
    fast = fast && transport_fast_set(sets[i]);
  }
  for (int i = 0; i < n; ++i) {
    const SetDesc& d = sets[i];
    smem = std::max(smem, set_smem(d, hm));
  }
  if (smem > (size_t)c->max_smem) return fail(PDV_EINVAL, "batch tables need %zu bytes of shared memory", smem);
  int grid = 0, block = 0;
  pdv_status s = f32_geometry(c, smem, hm, dump, impl, fast, &grid, &block);
  if (s != PDV_OK) return s;
  const std::string key = batch_key(c, rs, n, grid, block, smem, hm, dump) + (fast ? "f" : "g");
  pdv_ctx::GraphEntry* ge = nullptr;
  for (auto& g : c->graphs)
    if (g.key == key) ge = &g;
  const BatchLayout B = plan_batch(rs, n);
  if (!ge) {
    if (c->graphs.size() >= 8) {   // small LRU: drop the oldest
      auto& old = c->graphs.front();
      cudaStreamSynchronize(st);
      if (old.exec) cudaGraphExecDestroy(old.exec);
      ctx_free(c, old.arena, st);
      if (old.pinned) cudaFreeHost(old.pinned);
      cudaStreamSynchronize(st);
      c->graphs.erase(c->graphs.begin());
    }
    pdv_ctx::GraphEntry e;
    e.key = key;
    e.arena_bytes = B.bytes;
    e.arena = ctx_alloc(c, B.bytes, st);
    if (!e.arena) return fail(PDV_ENOMEM, "batch arena of %zu bytes failed", B.bytes);
    CK(cudaStreamSynchronize(st));
    char* base = (char*)e.arena;
    // capture the device work of the batch
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      cudaMemsetAsync(base + B.o_ctr, 0, sizeof(unsigned long long) * n, cap);
      cudaMemsetAsync(base + B.o_cnt, 0, sizeof(unsigned long long) * C_NCOUNT * n, cap);
      cudaMemsetAsync(base + B.o_hist, 0, sizeof(unsigned long long) * B.hist_words, cap);
      cudaEventRecordWithFlags(c->ev0, cap, cudaEventRecordExternal);
      launch_transport_f32((const SetDesc*)(base + B.o_sets), n,
                           (unsigned long long*)(base + B.o_ctr), grid, block, smem, hm, dump, impl,
                           fast, (unsigned)c->tuning.tile_packets, cap);
      cudaEventRecordWithFlags(c->ev1, cap, cudaEventRecordExternal);
      int max_snap = 1;
      for (int i = 0; i < n; ++i) max_snap = std::max(max_snap, rs[i].n_snap);
      launch_normalise((const SetDesc*)(base + B.o_sets), n, (double* const*)(base + B.o_pspec),
                       (pdv_counters* const*)(base + B.o_pcnt),
                       (unsigned long long* const*)(base + B.o_praw),
                       (const unsigned*)(base + B.o_flags), max_snap, cap);
      ce = cudaStreamEndCapture(cap, &graph);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess) {
      ctx_free(c, e.arena, st);
      cudaStreamSynchronize(st);
      return fail(PDV_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(ce));
    }
    c->graphs.push_back(e);
    ge = &c->graphs.back();
  }
  char* base = (char*)ge->arena;
  // per-call uploads: descriptors, snapshot times, output pointers, flags
  std::vector<double> ts;
  std::vector<void*> pspec(n), pcnt(n), praw(n);
  std::vector<unsigned> flags(n);
  for (int i = 0; i < n; ++i) {
    const pdv_request& r = rs[i];
    const bool dev = (r.flags & PDV_OUT_DEVICE) != 0;
    SetDesc& d = sets[i];
    d.t_snap = (const double*)(base + B.o_t_i[i]);
    d.hist = (unsigned long long*)(base + B.o_hist_i[i]);
    d.cnt = (unsigned long long*)(base + B.o_cnt) + (size_t)C_NCOUNT * i;
    d.packets = r.out_packets ? (dev ? r.out_packets : (pdv_packet_record*)(base + B.o_pk_i[i])) : nullptr;
    const size_t at = ts.size();
    ts.resize(at + time_words(r.n_snap));
    fill_times(&r, ts.data() + at);
    pspec[i] = dev ? (void*)r.out_spectrum : (void*)(base + B.o_spec_i[i]);
    pcnt[i] = r.out_counters ? (dev ? (void*)r.out_counters : (void*)(base + B.o_cout_i[i])) : nullptr;
    praw[i] = r.out_raw ? (dev ? (void*)r.out_raw : (void*)(base + B.o_raw_i[i])) : nullptr;
    flags[i] = r.flags;
  }
  CK(cudaMemcpyAsync(base + B.o_sets, sets.data(), sizeof(SetDesc) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + B.o_t, ts.data(), sizeof(double) * ts.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + B.o_pspec, pspec.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + B.o_pcnt, pcnt.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + B.o_praw, praw.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + B.o_flags, flags.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice, st));
  CK(cudaGraphLaunch(ge->exec, st));
  c->launches += 2;
  c->last_grid = grid;
  c->last_block = block;
  c->last_fast = fast && !dump;
  for (int i = 0; i < n; ++i) {
    const pdv_request& r = rs[i];
    if (r.flags & PDV_OUT_DEVICE) continue;
    CK(cudaMemcpyAsync(r.out_spectrum, pspec[i], sizeof(double) * (size_t)r.n_snap * r.n_bins, cudaMemcpyDeviceToHost, st));
    if (r.out_counters) CK(cudaMemcpyAsync(r.out_counters, pcnt[i], sizeof(pdv_counters) * r.n_snap, cudaMemcpyDeviceToHost, st));
    if (r.out_raw) CK(cudaMemcpyAsync(r.out_raw, praw[i], sizeof(unsigned long long) * (size_t)r.n_snap * (r.n_bins + 2), cudaMemcpyDeviceToHost, st));
    if (r.out_packets) CK(cudaMemcpyAsync(r.out_packets, base + B.o_pk_i[i], sizeof(pdv_packet_record) * r.n_packets, cudaMemcpyDeviceToHost, st));
  }
  std::vector<unsigned long long> cnts((size_t)C_NCOUNT * n);
  CK(cudaMemcpyAsync(cnts.data(), base + B.o_cnt, sizeof(unsigned long long) * cnts.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  unsigned long long ev = 0;
  for (int i = 0; i < n; ++i) ev += cnts[(size_t)C_NCOUNT * i + C_EVENTS];
  c->last_events = ev;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) {
    c->last_transport_ms = ms;
    if (transport_ms) *transport_ms = ms;
  }
  cudaGetLastError();
  (void)timed;
  return PDV_OK;
}

extern "C" pdv_status pdv_simulate_batch(pdv_ctx* c, const pdv_request* rs, int n) {
  NvtxRange nvtx_range("pdv_simulate_batch");
  if (!c || !rs || n < 1) return fail(PDV_EINVAL, "need a context and n >= 1 requests");
  for (int i = 0; i < n; ++i) {
    pdv_status s = validate_request(&rs[i]);
    if (s != PDV_OK) return fail(s, "request %d: %s", i, g_err.c_str());
    if (rs[i].n_layers)
      return fail(PDV_EINVAL, "request %d: layer stepping runs through pdv_simulate_spectrum only", i);
  }
  std::vector<pdv_request> f32;
  for (int i = 0; i < n; ++i) {
    if (rs[i].precision == PDV_PREC_FP32) f32.push_back(rs[i]);
    else {
      pdv_status s = pdv_simulate_spectrum(c, &rs[i]);
      if (s != PDV_OK) return s;
    }
  }
  if (f32.empty()) return PDV_OK;
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  const pdv_status s = run_batch_f32(c, f32.data(), (int)f32.size(), true, nullptr);
  return s != PDV_OK ? s : debug_after(c);
}

// ------------------------------------------------------------------ issue-rate probe
namespace pdv {
// Eight independent chains of FP32 fused multiply-adds per thread, 64 per loop
// trip: with 64 warps per SM every scheduler has a ready instruction each
// cycle, so the FMA count per second is the SM's sustained issue rate (one
// warp instruction per scheduler per cycle) at the clock the GPU runs.
__device__ float g_issue_sink[1];

__global__ void __launch_bounds__(256) k_issue_probe(int iters, float m, float a) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], m, a);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == -1.0f) g_issue_sink[0] = s;           // never true (x stays > 0): keeps the chains live
}
}  // namespace pdv

extern "C" pdv_status pdv_measure_issue_rate(pdv_ctx* c, double seconds, double* out) {
  NvtxRange nvtx_range("pdv_measure_issue_rate");
  if (!c || !out) return fail(PDV_EINVAL, "ctx and out must not be NULL");
  if (!(seconds > 0.0) || seconds > 10.0) return fail(PDV_EINVAL, "seconds must be in (0, 10]");
  std::lock_guard<std::mutex> lk(c->mu);
  CK(cudaSetDevice(c->device));
  const int grid = c->sm_count * 8, block = 256;
  auto run = [&](int iters, float* ms) -> pdv_status {
    CK(cudaEventRecord(c->ev0, c->stream));
    k_issue_probe<<<grid, block, 0, c->stream>>>(iters, 0.999999f, 1e-7f);
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->ev1, c->stream));
    CK(cudaEventSynchronize(c->ev1));
    CK(cudaEventElapsedTime(ms, c->ev0, c->ev1));
    return PDV_OK;
  };
  float ms = 0.0f;
  pdv_status s = run(64, &ms);                         // warm-up and calibration
  if (s != PDV_OK) return s;
  const double per_iter = std::max((double)ms, 1e-3) / 64.0;
  const int iters = (int)std::min(2.0e6, std::max(256.0, seconds * 1e3 / per_iter));
  s = run(iters, &ms);
  if (s != PDV_OK) return s;
  c->launches += 2;
  const double fmas = (double)grid * block * (double)iters * 64.0;
  *out = fmas / (ms * 1e-3);
  return PDV_OK;
}

// Autotune cache: a flat JSON object {"key": {"block_threads": b, "blocks_per_sm": s,
// "tile_packets": t, "hist_mode": h, "ms": m}, ...}, written and read only here.
static std::string tune_key(const pdv_ctx* c, const pdv_request* rs, int n) {
  unsigned long long pk = 0;
  int snap = 0, bins = 0;
  unsigned flags = 0;
  for (int i = 0; i < n; ++i) {
    pk += rs[i].n_packets;
    snap = std::max(snap, rs[i].n_snap);
    bins = std::max(bins, rs[i].n_bins);
    flags |= rs[i].flags & PDV_IMPLICIT_CAPTURE;
    if (rs[i].probe.aperture_radius_mm <= 0) flags |= 0x100u;
  }
  std::string name = c->device_name;
  for (char& ch : name)
    if (ch == '"' || ch == '\\' || ch == '|') ch = '_';
  char buf[320];
  snprintf(buf, sizeof buf, "%s|%d|%d|%.1e|%d|%d|%x", name.c_str(), c->sm_count, n, (double)pk,
           snap, bins, flags);
  return buf;
}

static bool tune_cache_find(const std::string& text, const std::string& key, pdv_tuning* t) {
  const std::string q = "\"" + key + "\"";
  const size_t at = text.find(q);
  if (at == std::string::npos) return false;
  const size_t open = text.find('{', at + q.size()), close = text.find('}', at + q.size());
  if (open == std::string::npos || close == std::string::npos || close < open) return false;
  const std::string body = text.substr(open, close - open);
  auto field = [&](const char* f, int* v) {
    const size_t p = body.find(std::string("\"") + f + "\"");
    if (p == std::string::npos) return false;
    const size_t colon = body.find(':', p);
    return colon != std::string::npos && sscanf(body.c_str() + colon + 1, "%d", v) == 1;
  };
  pdv_tuning r{};
  if (!field("block_threads", &r.block_threads) || !field("blocks_per_sm", &r.blocks_per_sm) ||
      !field("tile_packets", &r.tile_packets) || !field("hist_mode", &r.hist_mode))
    return false;
  *t = r;
  return true;
}

static std::string read_file(const std::string& path) {
  std::string out;
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return out;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) out.append(buf, k);
  fclose(f);
  return out;
}

static std::mutex g_tune_file_mu;

extern "C" pdv_status pdv_set_autotune_cache(pdv_ctx* c, const char* path) {
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  c->tune_cache = path ? path : "";
  return PDV_OK;
}

extern "C" pdv_status pdv_autotune(pdv_ctx* c, const pdv_request* rs, int n, pdv_tuning* out) {
  NvtxRange nvtx_range("pdv_autotune");
  if (!c || !rs || n < 1) return fail(PDV_EINVAL, "need a context and n >= 1 requests");
  for (int i = 0; i < n; ++i) {
    pdv_status s = validate_request(&rs[i]);
    if (s != PDV_OK) return fail(s, "request %d: %s", i, g_err.c_str());
    if (rs[i].precision != PDV_PREC_FP32 || rs[i].n_layers)
      return fail(PDV_EINVAL, "autotune takes FP32 exact-free-path requests");
  }
  CK(enter(c->device));
  const std::string key = tune_key(c, rs, n);
  std::string cache;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    cache = c->tune_cache;
  }
  if (!cache.empty()) {
    std::lock_guard<std::mutex> fl(g_tune_file_mu);
    pdv_tuning t{};
    if (tune_cache_find(read_file(cache), key, &t)) {
      std::lock_guard<std::mutex> lk(c->mu);
      c->tuning = t;
      if (!c->tuning.block_threads) c->tuning.block_threads = 256;
      if (out) *out = c->tuning;
      return PDV_OK;
    }
  }
  // a shortened copy of the batch (1/16 of the packets, at least 65536 each)
  std::vector<pdv_request> shortb(rs, rs + n);
  std::vector<std::vector<double>> specs(n);
  for (int i = 0; i < n; ++i) {
    pdv_request& r = shortb[i];
    r.n_packets = std::max<unsigned long long>(std::min<unsigned long long>(r.n_packets, 65536),
                                               r.n_packets / 16);
    specs[i].resize((size_t)r.n_snap * r.n_bins);
    r.out_spectrum = specs[i].data();
    r.out_raw = nullptr;
    r.out_counters = nullptr;
    r.out_packets = nullptr;
    r.flags &= ~PDV_OUT_DEVICE;
  }
  pdv_tuning best{};
  float best_ms = 1e30f;
  const int blocks[] = {128, 256};
  const int modes[] = {1, 2};
  const int bps[] = {0, 2};
  const int chunks[] = {32, 64, 256};
  std::lock_guard<std::mutex> lk(c->mu);
  const pdv_tuning saved = c->tuning;
  best = saved;
  for (int bt : blocks)
    for (int hm : modes)
      for (int b : bps)
        for (int ch : chunks) {
          pdv_tuning t{};
          t.block_threads = bt;
          t.hist_mode = hm;
          t.blocks_per_sm = b;
          t.tile_packets = ch;
          c->tuning = t;
          float ms = 0.f, total = 0.f;
          bool ok = true;
          for (int rep = 0; rep < 3 && ok; ++rep) {
            if (run_batch_f32(c, shortb.data(), n, true, &ms) != PDV_OK) ok = false;
            if (rep) total += ms;        // first run warms up (and captures the graph)
          }
          if (ok && total < best_ms) {
            best_ms = total;
            best = t;
          }
        }
  c->tuning = best;
  if (out) *out = best;
  if (!cache.empty()) {
    // read-modify-write of the whole file: add this key's entry before the final '}'
    std::lock_guard<std::mutex> fl(g_tune_file_mu);
    std::string text = read_file(cache);
    const size_t last = text.rfind('}');
    char entry[512];
    snprintf(entry, sizeof entry,
             "\"%s\": {\"block_threads\": %d, \"blocks_per_sm\": %d, \"tile_packets\": %d, "
             "\"hist_mode\": %d, \"ms\": %.4f}", key.c_str(), best.block_threads, best.blocks_per_sm,
             best.tile_packets, best.hist_mode, best_ms / 2.0);
    if (last == std::string::npos || text.find('"') == std::string::npos)
      text = std::string("{\n  ") + entry + "\n}\n";
    else
      text = text.substr(0, last) + ",\n  " + entry + "\n}\n";
    const std::string tmp = cache + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f || fwrite(text.data(), 1, text.size(), f) != text.size()) {
      if (f) fclose(f);
      return fail(PDV_EINVAL, "cannot write the autotune cache %s", cache.c_str());
    }
    fclose(f);
    if (rename(tmp.c_str(), cache.c_str()) != 0)
      return fail(PDV_EINVAL, "cannot replace the autotune cache %s", cache.c_str());
  }
  return PDV_OK;
}

// ------------------------------------------------------------------ serving
// Continuous batching: admitted requests are cut into slices of up to
// `quantum` packets; every launch of the persistent kernel carries one slice
// of each active request (up to kMaxLaunchSets), so new requests join at the
// next launch and their work overlaps with the others' on the device. Slices
// add into the request's own integer histogram, so a request's result is the
// same alone and in the mix.
constexpr int kMaxLaunchSets = 256;
constexpr int kSlots = 3;

struct Request {
  pdv_ticket id = 0;
  pdv_request req{};
  std::vector<double> ts;
  char* arena = nullptr;
  ReqBuffers b{};
  SetDesc d{};
  unsigned long long next = 0, done = 0;
  int state = 0;                     // 0 running, 1 finalising, 2 done, 3 failed/cancelled
  pdv_status status = PDV_OK;
  std::string err;
  bool cancelled = false;
  cudaEvent_t fin = nullptr;
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  size_t o_spec = 0, o_cnt = 0, o_raw = 0;
};

struct LaunchSlot {
  SetDesc* h_sets = nullptr;         // pinned
  char* d_mem = nullptr;             // SetDesc[kMaxLaunchSets] + counters[kMaxLaunchSets]
  cudaEvent_t ev = nullptr;
  std::vector<std::pair<std::shared_ptr<Request>, unsigned long long>> items;
  bool busy = false;
};

static void finish_request(pdv_ctx* c, const std::shared_ptr<Request>& q) {
  // normalise and stage the outputs into pinned memory on the serving stream
  NvtxRange nvtx_range("pdv serving normalise");
  const pdv_request& r = q->req;
  char* base = q->arena;
  const bool dev = (r.flags & PDV_OUT_DEVICE) != 0;
  launch_normalise((const SetDesc*)(base + q->b.o_set), 1, (double* const*)(base + q->b.o_ptr_spec),
                   (pdv_counters* const*)(base + q->b.o_ptr_cnt),
                   (unsigned long long* const*)(base + q->b.o_ptr_raw),
                   (const unsigned*)(base + q->b.o_flags), r.n_snap, c->serve_stream);
  c->launches += 1;
  if (!dev) {
    char* pin = (char*)q->pinned;
    cudaMemcpyAsync(pin + q->o_spec, base + q->b.o_spec, sizeof(double) * (size_t)r.n_snap * r.n_bins, cudaMemcpyDeviceToHost, c->serve_stream);
    if (r.out_counters) cudaMemcpyAsync(pin + q->o_cnt, base + q->b.o_cout, sizeof(pdv_counters) * r.n_snap, cudaMemcpyDeviceToHost, c->serve_stream);
    if (r.out_raw) cudaMemcpyAsync(pin + q->o_raw, base + q->b.o_craw, sizeof(unsigned long long) * (size_t)r.n_snap * (r.n_bins + 2), cudaMemcpyDeviceToHost, c->serve_stream);
  }
  cudaEventRecord(q->fin, c->serve_stream);
  q->state = 1;
}

static void complete_request(pdv_ctx* c, const std::shared_ptr<Request>& q) {
  const pdv_request& r = q->req;
  if (!(r.flags & PDV_OUT_DEVICE)) {
    const char* pin = (const char*)q->pinned;
    memcpy(r.out_spectrum, pin + q->o_spec, sizeof(double) * (size_t)r.n_snap * r.n_bins);
    if (r.out_counters) memcpy(r.out_counters, pin + q->o_cnt, sizeof(pdv_counters) * r.n_snap);
    if (r.out_raw) memcpy(r.out_raw, pin + q->o_raw, sizeof(unsigned long long) * (size_t)r.n_snap * (r.n_bins + 2));
  }
  ctx_free(c, q->arena, c->serve_stream);
  q->arena = nullptr;
  q->state = 2;
}

static void serving_loop(pdv_ctx* c) {
  enter(c->device);
  std::vector<LaunchSlot> slots(kSlots);
  for (auto& s : slots) {
    cudaMallocHost((void**)&s.h_sets, sizeof(SetDesc) * kMaxLaunchSets);
    cudaMalloc((void**)&s.d_mem, sizeof(SetDesc) * kMaxLaunchSets + sizeof(unsigned long long) * kMaxLaunchSets);
    cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
  }
  std::deque<int> inflight;
  std::vector<std::shared_ptr<Request>> finalising;
  size_t rr = 0;
  for (;;) {
    // 1. retire finished launches
    while (!inflight.empty()) {
      LaunchSlot& s = slots[inflight.front()];
      const bool must_wait = inflight.size() >= (size_t)kSlots;
      cudaError_t q = must_wait ? cudaEventSynchronize(s.ev) : cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) break;
      std::lock_guard<std::mutex> lk(c->smu);
      for (auto& it : s.items) {
        it.first->done += it.second;
        if (it.first->state == 3 && it.first->done == it.first->next && it.first->arena) {
          ctx_free(c, it.first->arena, c->serve_stream);   // cancelled or failed: last slice retired
          it.first->arena = nullptr;
        }
        if (q != cudaSuccess && it.first->state == 0) {
          it.first->state = 3;
          it.first->status = PDV_ECUDA;
          it.first->err = cudaGetErrorString(q);
        }
        if (it.first->state == 0 && it.first->done == it.first->req.n_packets) {
          finish_request(c, it.first);
          finalising.push_back(it.first);
        }
      }
      s.items.clear();
      s.busy = false;
      inflight.pop_front();
      c->done_cv.notify_all();
    }
    // 2. complete finalised requests
    for (size_t i = 0; i < finalising.size();) {
      if (cudaEventQuery(finalising[i]->fin) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(c->smu);
        complete_request(c, finalising[i]);
        finalising.erase(finalising.begin() + i);
        c->done_cv.notify_all();
      } else {
        ++i;
      }
    }
    // 3. build the next launch from the active requests
    int free_slot = -1;
    for (int k = 0; k < kSlots; ++k)
      if (!slots[k].busy) { free_slot = k; break; }
    std::vector<std::pair<std::shared_ptr<Request>, unsigned long long>> items;
    {
      std::unique_lock<std::mutex> lk(c->smu);
      // drop cancelled / finished requests from the active list
      for (size_t i = 0; i < c->active.size();) {
        auto& q = c->active[i];
        if (q->cancelled || q->next >= q->req.n_packets) c->active.erase(c->active.begin() + i);
        else ++i;
      }
      if (c->stop && c->active.empty() && inflight.empty() && finalising.empty()) break;
      if (free_slot >= 0 && !c->active.empty()) {
        const size_t na = c->active.size();
        for (size_t k = 0; k < na && (int)items.size() < kMaxLaunchSets; ++k) {
          auto& q = c->active[(rr + k) % na];
          const unsigned long long left = q->req.n_packets - q->next;
          const unsigned long long slice = std::min(left, c->quantum);
          items.emplace_back(q, slice);
        }
        rr += items.size();
      } else if (inflight.empty() && finalising.empty()) {
        c->scv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      for (auto& it : items) it.first->next += it.second;
    }
    if (items.empty()) {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      continue;
    }
    NvtxRange nvtx_launch("pdv serving launch");
    LaunchSlot& s = slots[free_slot];
    for (size_t k = 0; k < items.size(); ++k) {
      const auto& q = items[k].first;
      SetDesc d = q->d;
      d.packet_begin = q->req.packet_begin + (q->next - items[k].second);
      d.n_packets = items[k].second;
      s.h_sets[k] = d;
    }
    const int n = (int)items.size();
    size_t smem = 0;
    int hm = 1;
    bool impl = false, fast = true;
    for (int k = 0; k < n; ++k) {
      const SetDesc& d = s.h_sets[k];
      smem = std::max(smem, set_smem(d, 1));
      impl = impl || d.implicit != 0;
      fast = fast && transport_fast_set(d);
    }
    int grid = 0, block = 0;
    if (f32_geometry(c, smem, hm, false, impl, fast, &grid, &block) != PDV_OK) {
      std::lock_guard<std::mutex> lk(c->smu);
      for (auto& it : items) {
        it.first->state = 3;
        it.first->status = PDV_EINVAL;
        it.first->err = "request tables do not fit in shared memory";
      }
      c->done_cv.notify_all();
      continue;
    }
    cudaMemcpyAsync(s.d_mem, s.h_sets, sizeof(SetDesc) * n, cudaMemcpyHostToDevice, c->serve_stream);
    unsigned long long* ctr = (unsigned long long*)(s.d_mem + sizeof(SetDesc) * kMaxLaunchSets);
    cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * n, c->serve_stream);
    launch_transport_f32((const SetDesc*)s.d_mem, n, ctr, grid, block, smem, hm, false, impl, fast,
                         (unsigned)c->tuning.tile_packets, c->serve_stream);
    c->launches += 1;
    cudaEventRecord(s.ev, c->serve_stream);
    s.items = std::move(items);
    s.busy = true;
    inflight.push_back(free_slot);
  }
  for (auto& s : slots) {
    cudaFreeHost(s.h_sets);
    cudaFree(s.d_mem);
    cudaEventDestroy(s.ev);
  }
}

static pdv_status serving_start(pdv_ctx* c) {
  if (c->worker.joinable()) return PDV_OK;
  CK(cudaStreamCreateWithFlags(&c->serve_stream, cudaStreamNonBlocking));
  c->stop = false;
  c->worker = std::thread(serving_loop, c);
  return PDV_OK;
}

static void serving_stop(pdv_ctx* c) {
  if (!c->worker.joinable()) return;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    c->stop = true;
  }
  c->scv.notify_all();
  c->worker.join();
  for (auto& kv : c->requests) {
    auto& q = kv.second;
    if (q->arena) ctx_free(c, q->arena, c->serve_stream);
    if (q->fin) cudaEventDestroy(q->fin);
    pin_release(c, q->pinned, q->pinned_bytes);
  }
  c->requests.clear();
  cudaStreamSynchronize(c->serve_stream);
  cudaStreamDestroy(c->serve_stream);
  c->serve_stream = nullptr;
}

extern "C" pdv_status pdv_submit(pdv_ctx* c, const pdv_request* r, pdv_ticket* out) {
  NvtxRange nvtx_range("pdv_submit");
  if (!c || !out) return fail(PDV_EINVAL, "NULL argument");
  pdv_status s = validate_request(r);
  if (s != PDV_OK) return s;
  if (r->n_layers) return fail(PDV_EINVAL, "layer stepping runs through pdv_simulate_spectrum only");
  if (r->precision != PDV_PREC_FP32) return fail(PDV_EINVAL, "serving runs FP32 requests");
  if (r->out_packets) return fail(PDV_EINVAL, "serving does not dump packets");
  CK(enter(c->device));
  s = serving_start(c);
  if (s != PDV_OK) return s;
  const bool dev = (r->flags & PDV_OUT_DEVICE) != 0;
  auto q = std::make_shared<Request>();
  q->req = *r;
  q->ts.resize(time_words(r->n_snap));
  fill_times(r, q->ts.data());
  q->b = plan_request(r, dev);
  {
    std::lock_guard<std::mutex> lk(c->smu);
    if ((int)c->requests.size() >= c->max_slots)
      return fail(PDV_EAGAIN, "all %d request slots are in use", c->max_slots);
  }
  // admission by free device memory (keeping mem_reserve free, 256 MiB by
  // default); the driver is asked at most every 20 ms and the bytes admitted
  // since are subtracted
  {
    std::lock_guard<std::mutex> lk(c->smu);
    const auto now = std::chrono::steady_clock::now();
    if (now - c->mem_checked > std::chrono::milliseconds(20)) {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      c->mem_free = fr;
      c->mem_checked = now;
    }
    if (c->mem_free < q->b.bytes || c->mem_free - q->b.bytes < c->mem_reserve)
      return fail(PDV_EAGAIN, "not enough free device memory (%zu bytes free, %zu needed + %llu kept free)",
                  c->mem_free, q->b.bytes, (unsigned long long)c->mem_reserve);
    c->mem_free -= q->b.bytes;
  }
  q->arena = (char*)ctx_alloc(c, q->b.bytes, c->serve_stream);
  if (!q->arena) return fail(PDV_EAGAIN, "request allocation failed");
  char* base = q->arena;
  SetDesc d = make_set(r);
  d.t_snap = (const double*)(base + q->b.o_t);
  d.hist = (unsigned long long*)(base + q->b.o_hist);
  d.cnt = (unsigned long long*)(base + q->b.o_cnt);
  d.packets = nullptr;
  q->d = d;
  double* spec = dev ? r->out_spectrum : (double*)(base + q->b.o_spec);
  pdv_counters* cout = r->out_counters ? (dev ? r->out_counters : (pdv_counters*)(base + q->b.o_cout)) : nullptr;
  unsigned long long* raw = r->out_raw ? (dev ? (unsigned long long*)r->out_raw : (unsigned long long*)(base + q->b.o_craw)) : nullptr;
  const unsigned flags = r->flags;
  cudaStream_t st = c->serve_stream;
  // one pinned buffer per request: the uploads below (copied from pinned
  // memory, so the driver never has to wait for the serving stream) and,
  // for host outputs, the staged results
  Layout L;
  const size_t o_up_set = L.add(sizeof(SetDesc));
  const size_t o_up_t = L.add(sizeof(double) * time_words(r->n_snap));
  const size_t o_up_ptr = L.add(sizeof(void*) * 3 + sizeof(unsigned));
  q->o_spec = dev ? 0 : L.add(sizeof(double) * (size_t)r->n_snap * r->n_bins);
  q->o_cnt = (!dev && r->out_counters) ? L.add(sizeof(pdv_counters) * r->n_snap) : 0;
  q->o_raw = (!dev && r->out_raw) ? L.add(sizeof(unsigned long long) * (size_t)r->n_snap * (r->n_bins + 2)) : 0;
  q->pinned = pin_acquire(c, L.bytes, &q->pinned_bytes);
  if (!q->pinned) {
    ctx_free(c, q->arena, c->serve_stream);
    return fail(PDV_EAGAIN, "pinned staging allocation failed");
  }
  char* pin = (char*)q->pinned;
  memcpy(pin + o_up_set, &q->d, sizeof(SetDesc));
  memcpy(pin + o_up_t, q->ts.data(), sizeof(double) * q->ts.size());
  void* ptrs[3] = {(void*)spec, (void*)cout, (void*)raw};
  memcpy(pin + o_up_ptr, ptrs, sizeof ptrs);
  memcpy(pin + o_up_ptr + sizeof ptrs, &flags, sizeof flags);
  CK(cudaEventCreateWithFlags(&q->fin, cudaEventDisableTiming));
  CK(cudaMemcpyAsync(base + q->b.o_t, pin + o_up_t, sizeof(double) * q->ts.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + q->b.o_set, pin + o_up_set, sizeof(SetDesc), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + q->b.o_ptr_spec, pin + o_up_ptr, sizeof(void*), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + q->b.o_ptr_cnt, pin + o_up_ptr + sizeof(void*), sizeof(void*), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + q->b.o_ptr_raw, pin + o_up_ptr + 2 * sizeof(void*), sizeof(void*), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + q->b.o_flags, pin + o_up_ptr + sizeof ptrs, sizeof flags, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(base + q->b.o_cnt, 0, sizeof(unsigned long long) * C_NCOUNT, st));
  CK(cudaMemsetAsync(base + q->b.o_hist, 0, sizeof(unsigned long long) * hist_row(r->n_bins) * r->n_snap, st));
  // (the worker's launches for this request follow these copies on the same stream)
  {
    std::lock_guard<std::mutex> lk(c->smu);
    q->id = c->next_ticket++;
    c->requests[q->id] = q;
    c->active.push_back(q);
  }
  c->scv.notify_all();
  *out = q->id;
  return PDV_OK;
}

extern "C" pdv_status pdv_set_serving_limits(pdv_ctx* c, int max_requests, uint64_t reserve_bytes) {
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  if (max_requests < 1 || max_requests > 65536) return fail(PDV_EINVAL, "max_requests must be in [1, 65536]");
  std::lock_guard<std::mutex> lk(c->smu);
  c->max_slots = max_requests;
  c->mem_reserve = reserve_bytes;
  return PDV_OK;
}

extern "C" pdv_status pdv_poll(pdv_ctx* c, pdv_ticket t, uint32_t timeout_us) {
  NvtxRange nvtx_range("pdv_poll");
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  std::unique_lock<std::mutex> lk(c->smu);
  auto it = c->requests.find(t);
  if (it == c->requests.end()) return fail(PDV_EINVAL, "unknown ticket %llu", (unsigned long long)t);
  std::shared_ptr<Request> q = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  while (q->state < 2) {
    if (c->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && q->state < 2)
      return fail(PDV_ENOTREADY, "request %llu still running", (unsigned long long)t);
  }
  pdv_status s = q->status;
  std::string err = q->err;
  if (q->state == 3 && q->arena && q->next <= q->done) {
    ctx_free(c, q->arena, c->serve_stream);
    q->arena = nullptr;
  }
  const bool in_flight = q->state == 3 && q->next > q->done;
  if (!in_flight) {
    if (q->fin) cudaEventDestroy(q->fin);
    pin_release(c, q->pinned, q->pinned_bytes);
    q->fin = nullptr;
    q->pinned = nullptr;
    c->requests.erase(it);
  }
  if (s != PDV_OK) return fail(s, "request %llu: %s", (unsigned long long)t, err.c_str());
  return PDV_OK;
}

extern "C" pdv_status pdv_cancel(pdv_ctx* c, pdv_ticket t) {
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lk(c->smu);
  auto it = c->requests.find(t);
  if (it == c->requests.end()) return fail(PDV_EINVAL, "unknown ticket %llu", (unsigned long long)t);
  auto& q = it->second;
  if (q->state == 0) {
    q->cancelled = true;
    q->state = 3;
    q->status = PDV_ECANCELLED;
    q->err = "cancelled";
  }
  c->done_cv.notify_all();
  return PDV_OK;
}

// ------------------------------------------------------------------ fixed scratch
// pdv_simulate_spectrum_static: the FP32 spectrum call for callers that may
// not allocate device memory at run time (for example code running under an
// external memory budget or allocator that forbids cudaMalloc after start-up,
// or a host that pre-plans every byte of device memory). Its scratch lives in
// this file-scope device array instead: every GPU that loads the library holds
// these 4 MiB until the process exits. Every call shares the array, so calls
// that overlap on the GPU (different streams or contexts on one device) race.
constexpr size_t kStaticScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// In host code g_static_scratch names a host-side stand-in, not device memory:
// pdv_ctx_create looks its device address up with the context's device
// current and keeps it in the context.
static cudaError_t static_scratch_lookup(char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  *out = (char*)p;
  if (e == cudaSuccess && !p) return cudaErrorInvalidSymbol;
  return e;
}

// Scratch layout: a 1024-byte slot for the set descriptor, four 256-byte
// slots (packet counter, event counters, normalisation pointers, flags), then
// the histogram and the snapshot times, each rounded up to 256 bytes:
//   2048 + ceil256(8 n_snap (n_bins + 3)) + ceil256(24 n_snap) <= 4 MiB.
static_assert(sizeof(SetDesc) <= 1024, "set descriptor slot");
static_assert(sizeof(unsigned long long) * C_NCOUNT <= 256, "counter slot");

static size_t ceil256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t static_scratch_bytes(int n_snap, int n_bins) {
  return 2048 + ceil256(sizeof(unsigned long long) * (size_t)hist_row(n_bins) * n_snap) +
         ceil256(sizeof(double) * time_words(n_snap));
}

extern "C" pdv_status pdv_simulate_spectrum_static(pdv_ctx* c, const pdv_request* r) {
  NvtxRange nvtx_range("pdv_simulate_spectrum_static");
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  pdv_status s = validate_request(r);
  if (s != PDV_OK) return s;
  if (r->n_layers) return fail(PDV_EINVAL, "layer stepping runs through pdv_simulate_spectrum only");
  if (r->precision != PDV_PREC_FP32) return fail(PDV_EINVAL, "the static-scratch call runs FP32 requests");
  if (!(r->flags & PDV_OUT_DEVICE)) return fail(PDV_EINVAL, "the static-scratch call needs PDV_OUT_DEVICE outputs");
  const size_t need = static_scratch_bytes(r->n_snap, r->n_bins);
  if (need > kStaticScratchBytes)
    return fail(PDV_EINVAL, "request needs %zu bytes of scratch (2048 + ceil256(8 n_snap (n_bins + 3)) "
                "+ ceil256(24 n_snap)); the static scratch holds %zu", need, kStaticScratchBytes);
  const size_t o_set = 0, o_ctr = 1024, o_cnt = 1280, o_ptr = 1536, o_flags = 1792, o_hist = 2048;
  const size_t hist_words = (size_t)hist_row(r->n_bins) * r->n_snap;
  const size_t o_t = o_hist + ceil256(sizeof(unsigned long long) * hist_words);
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  char* base = c->static_scratch;
  cudaStream_t st = c->stream;
  SetDesc d = make_set(r);
  d.t_snap = (const double*)(base + o_t);
  d.hist = (unsigned long long*)(base + o_hist);
  d.cnt = (unsigned long long*)(base + o_cnt);
  d.packets = r->out_packets;
  double* ts = c->static_ts.data();            // made with the context: no allocation here
  fill_times_into(r, ts, c->static_idx.data());
  void* ptrs[3] = {(void*)r->out_spectrum, (void*)r->out_counters, (void*)r->out_raw};
  const unsigned flags = r->flags;
  CK(cudaMemcpyAsync(base + o_t, ts, sizeof(double) * time_words(r->n_snap), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + o_set, &d, sizeof d, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + o_ptr, ptrs, sizeof ptrs, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + o_flags, &flags, sizeof flags, cudaMemcpyHostToDevice, st));
  // the previous call's counts stay in the array: clear what accumulates
  CK(cudaMemsetAsync(base + o_ctr, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(base + o_cnt, 0, sizeof(unsigned long long) * C_NCOUNT, st));
  CK(cudaMemsetAsync(base + o_hist, 0, sizeof(unsigned long long) * hist_words, st));
  const int hm = pick_hist_mode(c, d);
  const bool dump = d.packets != nullptr;
  const size_t smem = set_smem(d, hm);
  if (smem > (size_t)c->max_smem) return fail(PDV_EINVAL, "tables need %zu bytes of shared memory", smem);
  int grid = 0, block = 0;
  const bool impl = d.implicit != 0;
  const bool fast = transport_fast_set(d);
  s = f32_geometry(c, smem, hm, dump, impl, fast, &grid, &block, true);
  if (s != PDV_OK) return s;
  launch_transport_f32_one(d, (unsigned long long*)(base + o_ctr), grid, block, smem, hm, dump, impl,
                           fast, (unsigned)c->tuning.tile_packets, st);
  c->last_fast = fast && !dump;
  launch_normalise((const SetDesc*)(base + o_set), 1, (double* const*)(base + o_ptr),
                   (pdv_counters* const*)(base + o_ptr + sizeof(void*)),
                   (unsigned long long* const*)(base + o_ptr + 2 * sizeof(void*)),
                   (const unsigned*)(base + o_flags), r->n_snap, st);
  c->launches += 2;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return debug_after(c);
}

// ------------------------------------------------------------------ spectrum model
// Single-scattering spectra (Eq. 22-28) and peak extraction (Eq. 29-35).
static bool ss_set_valid(const pdv_ss_set& s) {
  return s.beta > 0.0 && std::isfinite(s.beta) && s.tau0 >= 0.0 && std::isfinite(s.tau0) &&
         s.v_fs > 0.0 && std::isfinite(s.v_fs) && std::isfinite(s.prefactor) && !std::isnan(s.v_max);
}

extern "C" pdv_status pdv_ss_spectrum(pdv_ctx* c, const pdv_ss_set* sets, int n_sets, int n_bins,
                                      double v_lo, double v_hi, uint32_t flags, double* out) {
  NvtxRange nvtx_range("pdv_ss_spectrum");
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  if (n_sets < 0 || n_bins < 1) return fail(PDV_EINVAL, "n_sets must be >= 0 and n_bins >= 1");
  if (!(v_hi > v_lo) || !std::isfinite(v_lo) || !std::isfinite(v_hi))
    return fail(PDV_EINVAL, "need finite v_lo < v_hi");
  if (flags & ~(PDV_IN_DEVICE | PDV_OUT_DEVICE | PDV_PER_DV)) return fail(PDV_EINVAL, "unknown flags");
  if ((long long)n_sets * n_bins > (1LL << 36)) return fail(PDV_EINVAL, "n_sets * n_bins too large");
  if (n_sets == 0) return PDV_OK;
  if (!sets || !out) return fail(PDV_EINVAL, "sets and out must not be NULL");
  const bool dev_in = (flags & PDV_IN_DEVICE) != 0, dev_out = (flags & PDV_OUT_DEVICE) != 0;
  if (!dev_in)
    for (int i = 0; i < n_sets; ++i)
      if (!ss_set_valid(sets[i]))
        return fail(PDV_EINVAL, "set %d: need beta > 0, tau0 >= 0, v_fs > 0, finite values", i);
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t st = c->stream;
  const size_t out_bytes = sizeof(double) * (size_t)n_sets * n_bins;
  Layout L;
  const size_t o_sets = dev_in ? 0 : L.add(sizeof(pdv_ss_set) * (size_t)n_sets);
  const size_t o_const = L.add(ss_const_bytes() * (size_t)n_sets);
  const size_t o_bad = L.add(sizeof(int));
  const size_t o_out = dev_out ? 0 : L.add(out_bytes);
  char* base = (char*)ctx_alloc(c, L.bytes, st);
  if (!base) return fail(PDV_ENOMEM, "model allocation of %zu bytes failed", L.bytes);
  struct Guard {
    pdv_ctx* c; char* p; cudaStream_t st;
    ~Guard() { ctx_free(c, p, st); cudaStreamSynchronize(st); }
  } guard{c, base, st};
  const pdv_ss_set* d_sets = dev_in ? sets : (const pdv_ss_set*)(base + o_sets);
  double* d_out = dev_out ? out : (double*)(base + o_out);
  if (!dev_in)
    CK(cudaMemcpyAsync(base + o_sets, sets, sizeof(pdv_ss_set) * (size_t)n_sets, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(base + o_bad, 0, sizeof(int), st));
  CK(launch_ss_const(d_sets, n_sets, n_bins, v_lo, v_hi, (flags & PDV_PER_DV) ? 1 : 0,
                     base + o_const, (int*)(base + o_bad), st));
  CK(cudaEventRecord(c->ev0, st));
  CK(launch_ss_bins(base + o_const, n_sets, n_bins, d_out, st));
  CK(cudaEventRecord(c->ev1, st));
  c->launches += 2;
  if (!dev_out) CK(cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, st));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, base + o_bad, sizeof bad, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->last_model_ms = ms;
  cudaGetLastError();
  if (bad) return fail(PDV_EINVAL, "%d device-resident sets are invalid (their bins are NaN)", bad);
  return PDV_OK;
}

extern "C" pdv_status pdv_extract_peaks(pdv_ctx* c, const double* spectra, int n_spectra,
                                        int n_bins, double v_lo, double v_hi, double v_fs,
                                        const pdv_peak_opts* opts, uint32_t flags, pdv_peak* out) {
  NvtxRange nvtx_range("pdv_extract_peaks");
  if (!c || !opts) return fail(PDV_EINVAL, "ctx and opts must not be NULL");
  if (n_spectra < 0) return fail(PDV_EINVAL, "n_spectra must be >= 0");
  if (n_bins < 3 || n_bins > kPeakMaxBins) return fail(PDV_EINVAL, "n_bins must be in [3, %d]", kPeakMaxBins);
  if (opts->k_c < 1 || 2 * opts->k_c >= n_bins) return fail(PDV_EINVAL, "k_c must satisfy 1 <= k_c < n_bins / 2");
  if (!(v_hi > v_lo) || !std::isfinite(v_lo) || !std::isfinite(v_hi) || !(v_fs > 0.0) || !std::isfinite(v_fs))
    return fail(PDV_EINVAL, "need finite v_lo < v_hi and v_fs > 0");
  if (std::isnan(opts->x_min) || std::isnan(opts->x_max)) return fail(PDV_EINVAL, "window bounds are NaN");
  if (flags & ~(PDV_IN_DEVICE | PDV_OUT_DEVICE | PDV_EXTRACT_SIMT)) return fail(PDV_EINVAL, "unknown flags");
  if (n_spectra == 0) return PDV_OK;
  if (!spectra || !out) return fail(PDV_EINVAL, "spectra and out must not be NULL");
  const bool dev_in = (flags & PDV_IN_DEVICE) != 0, dev_out = (flags & PDV_OUT_DEVICE) != 0;
  // window: bin centres x_j = (v_lo + (j + 1/2) dv) / v_fs inside [x_min, x_max]
  const double dv = (v_hi - v_lo) / n_bins;
  int j_lo = n_bins, j_hi = -1;
  for (int j = 0; j < n_bins; ++j) {
    const double x = (v_lo + ((double)j + 0.5) * dv) / v_fs;
    if (x >= opts->x_min && j_lo == n_bins) j_lo = j;
    if (x <= opts->x_max) j_hi = j;
  }
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t st = c->stream;
  // the tensor-core kernel (128 spectra per block) where it fits, unless
  // PDV_EXTRACT_SIMT; else cut-offs up to 95 modes take the tiled kernel (64
  // spectra per block), larger ones the one-spectrum-per-block kernel
  const bool tc = !(flags & PDV_EXTRACT_SIMT) && peak_tc(opts->k_c, c->smem_optin);
  const bool tiled = !tc && peak_tiled(opts->k_c);
  int occ = 0;
  if (tc) CK(tc_occupancy(opts->k_c, &occ));
  else if (tiled) CK(tiled_occupancy(opts->k_c, &occ));
  else CK(peak_occupancy(n_bins, opts->k_c, &occ));
  if (occ < 1) return fail(PDV_EINVAL, "extraction tables do not fit in shared memory");
  const size_t in_bytes = sizeof(double) * (size_t)n_spectra * n_bins;
  const size_t out_bytes = sizeof(pdv_peak) * (size_t)n_spectra;
  Layout L;
  const size_t o_tw = L.add(sizeof(float2) * (size_t)n_bins);
  const size_t o_mats =
      tc ? L.add(peak_mats_tc_bytes(n_bins, opts->k_c, j_hi - j_lo + 1))
         : (tiled ? L.add(peak_mats_bytes(n_bins, opts->k_c, j_hi - j_lo + 1)) : 0);
  const size_t o_err = L.add(sizeof(int));
  const size_t o_in = dev_in ? 0 : L.add(in_bytes);
  const size_t o_out = dev_out ? 0 : L.add(out_bytes);
  char* base = (char*)ctx_alloc(c, L.bytes, st);
  if (!base) return fail(PDV_ENOMEM, "extraction allocation of %zu bytes failed", L.bytes);
  struct Guard {
    pdv_ctx* c; char* p; cudaStream_t st;
    ~Guard() { ctx_free(c, p, st); cudaStreamSynchronize(st); }
  } guard{c, base, st};
  const double* d_in = dev_in ? spectra : (const double*)(base + o_in);
  pdv_peak* d_out = dev_out ? out : (pdv_peak*)(base + o_out);
  if (!dev_in) CK(cudaMemcpyAsync(base + o_in, spectra, in_bytes, cudaMemcpyHostToDevice, st));
  CK(launch_twiddles(n_bins, (float2*)(base + o_tw), st));
  PeakGeom geom;
  geom.x0 = (float)((v_lo + 0.5 * dv) / v_fs);
  geom.dxj = (float)(dv / v_fs);
  geom.scale = (float)((v_fs / dv) * (v_fs / dv));
  int* d_err = (int*)(base + o_err);
  CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  if (tc) {
    CK(launch_extract_tc(d_in, n_spectra, n_bins, opts->k_c, j_lo, j_hi, geom,
                         (const float2*)(base + o_tw), (float*)(base + o_mats), d_out, d_err, occ,
                         c->sm_count, st, c->ev0, c->ev1));
    c->launches += 3;
  } else if (tiled) {
    CK(launch_extract_tiled(d_in, n_spectra, n_bins, opts->k_c, j_lo, j_hi, geom,
                            (const float2*)(base + o_tw), (float*)(base + o_mats), d_out, occ,
                            c->sm_count, st, c->ev0, c->ev1));
    c->launches += 3;
  } else {
    const int grid = (int)std::min<long long>((long long)occ * c->sm_count, n_spectra);
    CK(cudaEventRecord(c->ev0, st));
    CK(launch_extract(d_in, n_spectra, n_bins, opts->k_c, j_lo, j_hi, geom,
                      (const float2*)(base + o_tw), d_out, grid, st));
    CK(cudaEventRecord(c->ev1, st));
    c->launches += 2;
  }
  if (!dev_out) CK(cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, st));
  int err = 0;
  CK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->last_model_ms = ms;
  cudaGetLastError();
  if (err) return fail(PDV_ETIMEOUT, "tensor-core extraction: a wait for the products timed out");
  return PDV_OK;
}

// ------------------------------------------------------------------ debug build
extern "C" pdv_status pdv_debug_get(pdv_ctx* c, pdv_debug_info* out, int reset) {
  if (!c || !out) return fail(PDV_EINVAL, "ctx and out must not be NULL");
  memset(out, 0, sizeof *out);
  out->debug_build = kDebugBuild ? 1 : 0;
  if (!kDebugBuild) return PDV_OK;
  CK(enter(c->device));
  std::lock_guard<std::mutex> lk(c->mu);
  CK(cudaStreamSynchronize(c->stream));
  DebugWord a{}, b{};
  CK(transport_debug_io(&a, reset != 0, c->stream));
  CK(stepping_debug_io(&b, reset != 0, c->stream));
  const DebugWord& f = a.violations ? a : b;
  out->violations = a.violations + b.violations;
  if (f.violations) {
    out->site = f.site;
    out->index = f.index;
    out->bound = f.bound;
  }
  return PDV_OK;
}

extern "C" pdv_status pdv_debug_set_trace(pdv_ctx* c, int n_trace, int max_vertices,
                                          pdv_trace_vertex* out) {
  if (!c) return fail(PDV_EINVAL, "ctx is NULL");
  if (!kDebugBuild) return fail(PDV_EINVAL, "path traces need the debug build (libpdv_debug.so)");
  std::lock_guard<std::mutex> lk(c->mu);
  if (n_trace == 0) {
    c->trace_n = 0;
    c->trace_out = nullptr;
    return PDV_OK;
  }
  if (n_trace < 1 || n_trace > 65536 || max_vertices < 1 || max_vertices > 4096 || !out)
    return fail(PDV_EINVAL, "need 1 <= n_trace <= 65536, 1 <= max_vertices <= 4096 and an output array");
  c->trace_out = out;
  c->trace_n = n_trace;
  c->trace_max = max_vertices;
  return PDV_OK;
}
