"""Thin Python binding of libpdv (``include/pdv.h``): ctypes marshalling only.

Every step of the Monte Carlo runs in the library's CUDA kernels; there is no
Python or CPU fallback. If the shared library cannot be built or loaded, or no
CUDA device is present, the calls raise.

The library is ``libpdv.so``; with the environment variable
``PDV_LIBRARY=debug`` set before the first call, the process loads the debug
build ``libpdv_debug.so`` instead (index checks in the kernels, path traces).

Functions keep the C names (``pdv_ctx_create``, ``pdv_create_cloud``,
``pdv_set_phase_table``, ``pdv_simulate_spectrum``, ``pdv_simulate_batch``,
``pdv_submit``, ``pdv_poll``, ...). ``Context``, ``Cloud`` and
``simulate_spectrum`` are conveniences that convert a
:class:`~paper_2012_00963_gb300.workloads.Workload` (SI units) into the ABI's
units (mg/cm^2, um, nm, mm, us).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

PDV_OK, PDV_EINVAL, PDV_ENOMEM, PDV_ECUDA, PDV_EAGAIN = 0, -1, -2, -3, -4
PDV_ENOTREADY, PDV_ETIMEOUT, PDV_ECANCELLED, PDV_EDEBUG = -5, -6, -7, -8
PDV_OUT_DEVICE, PDV_PER_DV, PDV_IN_DEVICE, PDV_IMPLICIT_CAPTURE = 0x1, 0x2, 0x4, 0x8
PDV_TEST_HORIZONTAL_LAUNCH, PDV_TEST_DEBUG_CHECK, PDV_EXTRACT_SIMT = 0x10, 0x20, 0x40
DEBUG_SITES = ["none", "mass_guide", "mass_node", "phase_guide", "phase_node", "turn", "snapshot",
               "histogram", "packet", "selftest"]
PDV_PEAK_OK, PDV_PEAK_NO_PEAK, PDV_PEAK_NOT_MAX, PDV_PEAK_EDGE = 0, 1, 2, 3
PDV_PREC_FP32, PDV_PREC_FP64 = 0, 1
STATUS_NAMES = {0: "PDV_OK", -1: "PDV_EINVAL", -2: "PDV_ENOMEM", -3: "PDV_ECUDA",
                -4: "PDV_EAGAIN", -5: "PDV_ENOTREADY", -6: "PDV_ETIMEOUT", -7: "PDV_ECANCELLED",
                -8: "PDV_EDEBUG"}
COUNTER_NAMES = [
    "launched", "events", "scatters", "surface_hits", "escapes", "detected",
    "w_detected", "w_under", "w_over", "w_escaped_undetected", "w_absorbed_particle",
    "w_absorbed_surface", "w_truncated", "truncated", "w_roulette_dropped", "w_roulette_gained",
]
ABI_FUNCTIONS = [
    "pdv_ctx_create", "pdv_ctx_destroy", "pdv_last_error", "pdv_get_stats", "pdv_set_tuning",
    "pdv_create_cloud", "pdv_set_phase_table", "pdv_cloud_get_info", "pdv_destroy_cloud",
    "pdv_phase_hg", "pdv_mie_table", "pdv_simulate_spectrum", "pdv_simulate_batch",
    "pdv_autotune", "pdv_submit", "pdv_poll", "pdv_cancel", "pdv_simulate_spectrum_static",
    "pdv_ss_spectrum", "pdv_extract_peaks", "pdv_measure_issue_rate", "pdv_set_serving_limits",
    "pdv_set_autotune_cache", "pdv_debug_get", "pdv_debug_set_trace",
]


class PdvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


# ------------------------------------------------------------------ C structs
class pdv_allocator(C.Structure):
    _fields_ = [("alloc", C.c_void_p), ("free", C.c_void_p), ("user", C.c_void_p)]


class pdv_cloud_desc(C.Structure):
    _fields_ = [
        ("rho_kg_m3", C.c_double), ("area_mass_mg_cm2", C.c_double), ("v_fs", C.c_double),
        ("reflectivity", C.c_double), ("surface_mode", C.c_int), ("profile_kind", C.c_int),
        ("beta", C.c_double), ("v_max", C.c_double), ("prof_v", C.POINTER(C.c_double)),
        ("prof_dmdv", C.POINTER(C.c_double)), ("prof_n", C.c_int), ("d_median_um", C.c_double),
        ("sigma_ln", C.c_double), ("wavelength_nm", C.c_double), ("table_nodes", C.c_int),
    ]


class pdv_probe(C.Structure):
    _fields_ = [("z_probe_mm", C.c_double), ("beam_radius_mm", C.c_double),
                ("aperture_radius_mm", C.c_double), ("cone_half_angle_rad", C.c_double)]


class pdv_counters(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in COUNTER_NAMES]


PACKET_DTYPE = np.dtype([
    ("n_events", np.uint32), ("n_scatters", np.uint32), ("n_surface", np.uint32),
    ("fate", np.uint32), ("weight", np.uint64), ("v_app", np.float64),
    ("detect_mask", np.uint64),
])


class pdv_request(C.Structure):
    _fields_ = [
        ("cloud", C.c_void_p), ("probe", pdv_probe), ("t_snap_us", C.POINTER(C.c_double)),
        ("n_snap", C.c_int), ("n_packets", C.c_uint64), ("packet_begin", C.c_uint64),
        ("seed", C.c_uint64), ("stream_id", C.c_uint32), ("max_events", C.c_uint32),
        ("n_bins", C.c_int), ("v_lo", C.c_double), ("v_hi", C.c_double), ("precision", C.c_int),
        ("flags", C.c_uint32), ("out_spectrum", C.c_void_p), ("out_raw", C.c_void_p),
        ("out_counters", C.c_void_p), ("out_packets", C.c_void_p),
        ("n_layers", C.c_uint32), ("reserved", C.c_uint32),
    ]


class pdv_tuning(C.Structure):
    _fields_ = [("block_threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("tile_packets", C.c_int), ("hist_mode", C.c_int)]


class pdv_cloud_info(C.Structure):
    _fields_ = [("tau_tot", C.c_double), ("v_bot", C.c_double), ("v_top", C.c_double),
                ("d_sauter_um", C.c_double), ("g_table", C.c_double), ("q_ext", C.c_double),
                ("albedo", C.c_double), ("table_nodes", C.c_int), ("has_phase", C.c_int)]


class pdv_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("last_transport_ms", C.c_double),
                ("last_events", C.c_uint64), ("transport_grid", C.c_int),
                ("transport_block", C.c_int), ("last_model_ms", C.c_double),
                ("last_steps", C.c_uint64), ("transport_fast", C.c_int32), ("reserved", C.c_int32)]


class pdv_ss_set(C.Structure):
    _fields_ = [("beta", C.c_double), ("tau0", C.c_double), ("v_fs", C.c_double),
                ("v_max", C.c_double), ("prefactor", C.c_double)]


class pdv_peak_opts(C.Structure):
    _fields_ = [("k_c", C.c_int), ("reserved", C.c_int), ("x_min", C.c_double),
                ("x_max", C.c_double)]


class pdv_debug_info(C.Structure):
    _fields_ = [("debug_build", C.c_int32), ("site", C.c_uint32), ("violations", C.c_uint64),
                ("index", C.c_int64), ("bound", C.c_int64)]


TRACE_DTYPE = np.dtype([
    ("x", np.float64), ("y", np.float64), ("z", np.float64), ("v", np.float64),
    ("ux", np.float64), ("uy", np.float64), ("uz", np.float64), ("kind", np.int32),
    ("event", np.uint32),
])


class pdv_peak(C.Structure):
    _fields_ = [("x_peak", C.c_double), ("i_peak", C.c_double), ("curvature", C.c_double),
                ("beta", C.c_double), ("tau0", C.c_double), ("status", C.c_int32),
                ("j_max", C.c_int32)]


SS_SET_DTYPE = np.dtype([(f, np.float64) for f, _ in pdv_ss_set._fields_])
PEAK_DTYPE = np.dtype([("x_peak", np.float64), ("i_peak", np.float64), ("curvature", np.float64),
                       ("beta", np.float64), ("tau0", np.float64), ("status", np.int32),
                       ("j_max", np.int32)])


# ------------------------------------------------------------------ library
_lock = threading.Lock()
_lib = None


def debug_library() -> bool:
    """Whether this process loads the debug build (PDV_LIBRARY=debug)."""
    return os.environ.get("PDV_LIBRARY", "") == "debug"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_library() else _build.LIB


def lib():
    """Load libpdv.so (libpdv_debug.so under PDV_LIBRARY=debug), building it
    with nvcc first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=debug_library())
            L = C.CDLL(path)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
            sig = {
                "pdv_ctx_create": ([ip, vp, vp, C.POINTER(vp)], ip),
                "pdv_ctx_destroy": ([vp], ip),
                "pdv_last_error": ([], C.c_char_p),
                "pdv_get_stats": ([vp, C.POINTER(pdv_stats)], ip),
                "pdv_set_tuning": ([vp, C.POINTER(pdv_tuning)], ip),
                "pdv_create_cloud": ([vp, C.POINTER(pdv_cloud_desc), C.POINTER(vp)], ip),
                "pdv_set_phase_table": ([vp, ip, dp, dp, C.c_double, C.c_double], ip),
                "pdv_cloud_get_info": ([vp, C.POINTER(pdv_cloud_info)], ip),
                "pdv_destroy_cloud": ([vp], ip),
                "pdv_phase_hg": ([C.c_double, ip, dp, dp], ip),
                "pdv_mie_table": ([vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                   ip, ip, dp, dp, dp, dp, dp], ip),
                "pdv_simulate_spectrum": ([vp, C.POINTER(pdv_request)], ip),
                "pdv_simulate_batch": ([vp, C.POINTER(pdv_request), ip], ip),
                "pdv_simulate_spectrum_static": ([vp, C.POINTER(pdv_request)], ip),
                "pdv_autotune": ([vp, C.POINTER(pdv_request), ip, C.POINTER(pdv_tuning)], ip),
                "pdv_submit": ([vp, C.POINTER(pdv_request), C.POINTER(C.c_uint64)], ip),
                "pdv_poll": ([vp, C.c_uint64, C.c_uint32], ip),
                "pdv_cancel": ([vp, C.c_uint64], ip),
                "pdv_set_serving_limits": ([vp, ip, C.c_uint64], ip),
                "pdv_set_autotune_cache": ([vp, C.c_char_p], ip),
                "pdv_ss_spectrum": ([vp, vp, ip, ip, C.c_double, C.c_double, C.c_uint32, vp], ip),
                "pdv_extract_peaks": ([vp, vp, ip, ip, C.c_double, C.c_double, C.c_double,
                                       C.POINTER(pdv_peak_opts), C.c_uint32, vp], ip),
                "pdv_measure_issue_rate": ([vp, C.c_double, dp], ip),
                "pdv_debug_get": ([vp, C.POINTER(pdv_debug_info), ip], ip),
                "pdv_debug_set_trace": ([vp, ip, ip, vp], ip),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def last_error() -> str:
    m = lib().pdv_last_error()
    return m.decode() if m else ""


def _check(status):
    if status != PDV_OK:
        raise PdvError(status, last_error())
    return status


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------------ ABI (same names)
def pdv_ctx_create(device: int = 0, stream: Optional[int] = None,
                   allocator: Optional[pdv_allocator] = None) -> int:
    """``allocator``: a pdv_allocator whose callbacks the caller keeps alive
    for the context's lifetime (None: the context's own memory pool)."""
    h = C.c_void_p()
    _check(lib().pdv_ctx_create(device, C.c_void_p(stream or 0),
                                C.c_void_p(C.addressof(allocator)) if allocator is not None else None,
                                C.byref(h)))
    return h.value


def pdv_set_serving_limits(ctx: int, max_requests: int, reserve_bytes: int):
    _check(lib().pdv_set_serving_limits(C.c_void_p(ctx), int(max_requests), int(reserve_bytes)))


def pdv_ctx_destroy(ctx: int):
    _check(lib().pdv_ctx_destroy(C.c_void_p(ctx)))


def pdv_get_stats(ctx: int) -> dict:
    s = pdv_stats()
    _check(lib().pdv_get_stats(C.c_void_p(ctx), C.byref(s)))
    return {f: getattr(s, f) for f, _ in pdv_stats._fields_}


def pdv_set_tuning(ctx: int, block_threads=0, blocks_per_sm=0, tile_packets=0, hist_mode=0):
    t = pdv_tuning(block_threads, blocks_per_sm, tile_packets, hist_mode)
    _check(lib().pdv_set_tuning(C.c_void_p(ctx), C.byref(t)))


def pdv_create_cloud(ctx: int, desc: pdv_cloud_desc) -> int:
    h = C.c_void_p()
    _check(lib().pdv_create_cloud(C.c_void_p(ctx), C.byref(desc), C.byref(h)))
    return h.value


def pdv_set_phase_table(cloud: int, theta, p, q_ext_eff: float, albedo: float):
    th = np.ascontiguousarray(theta, np.float64)
    pp = np.ascontiguousarray(p, np.float64)
    if th.shape != pp.shape:
        raise ValueError("theta and p differ in length")
    _check(lib().pdv_set_phase_table(C.c_void_p(cloud), len(th), _dp(th), _dp(pp),
                                     float(q_ext_eff), float(albedo)))


def pdv_cloud_get_info(cloud: int) -> dict:
    i = pdv_cloud_info()
    _check(lib().pdv_cloud_get_info(C.c_void_p(cloud), C.byref(i)))
    return {f: getattr(i, f) for f, _ in pdv_cloud_info._fields_}


def pdv_destroy_cloud(cloud: int):
    _check(lib().pdv_destroy_cloud(C.c_void_p(cloud)))


def pdv_phase_hg(g: float, n: int = 1801):
    th = np.zeros(n)
    p = np.zeros(n)
    _check(lib().pdv_phase_hg(float(g), int(n), _dp(th), _dp(p)))
    return th, p


def pdv_mie_table(ctx: int, m: complex, wavelength_nm: float, d_median_um: float,
                  sigma_ln: float, n_size: int = 256, n_angle: int = 1801):
    th = np.zeros(n_angle)
    p = np.zeros(n_angle)
    q = np.zeros(3)
    _check(lib().pdv_mie_table(C.c_void_p(ctx), float(np.real(m)), float(np.imag(m)),
                               float(wavelength_nm), float(d_median_um), float(sigma_ln),
                               int(n_size), int(n_angle), _dp(th), _dp(p), _dp(q[0:1]),
                               _dp(q[1:2]), _dp(q[2:3])))
    return th, p, float(q[0]), float(q[1]), float(q[2])


def pdv_simulate_spectrum(ctx: int, req: pdv_request):
    _check(lib().pdv_simulate_spectrum(C.c_void_p(ctx), C.byref(req)))


def pdv_simulate_spectrum_static(ctx: int, req: pdv_request):
    """FP32 spectrum with the library's fixed device scratch (no allocation);
    outputs must be device buffers (PDV_OUT_DEVICE)."""
    _check(lib().pdv_simulate_spectrum_static(C.c_void_p(ctx), C.byref(req)))


def pdv_simulate_batch(ctx: int, reqs: Sequence[pdv_request]):
    arr = (pdv_request * len(reqs))(*reqs)
    _check(lib().pdv_simulate_batch(C.c_void_p(ctx), arr, len(reqs)))


def pdv_set_autotune_cache(ctx: int, path: Optional[str]):
    _check(lib().pdv_set_autotune_cache(C.c_void_p(ctx), path.encode() if path else None))


def pdv_autotune(ctx: int, reqs: Sequence[pdv_request]) -> dict:
    arr = (pdv_request * len(reqs))(*reqs)
    t = pdv_tuning()
    _check(lib().pdv_autotune(C.c_void_p(ctx), arr, len(reqs), C.byref(t)))
    return {f: getattr(t, f) for f, _ in pdv_tuning._fields_}


def pdv_measure_issue_rate(ctx: int, seconds: float = 0.2) -> float:
    """Measured FP32 FMA issue rate of the GPU, thread-instructions per second."""
    v = C.c_double()
    _check(lib().pdv_measure_issue_rate(C.c_void_p(ctx), float(seconds), C.byref(v)))
    return v.value


def pdv_submit(ctx: int, req: pdv_request) -> int:
    t = C.c_uint64()
    _check(lib().pdv_submit(C.c_void_p(ctx), C.byref(req), C.byref(t)))
    return t.value


def pdv_poll(ctx: int, ticket: int, timeout_us: int = 0) -> int:
    """PDV_OK when done, PDV_ENOTREADY while running; raises on errors."""
    s = lib().pdv_poll(C.c_void_p(ctx), C.c_uint64(ticket), C.c_uint32(timeout_us))
    if s in (PDV_OK, PDV_ENOTREADY):
        return s
    raise PdvError(s, last_error())


def pdv_cancel(ctx: int, ticket: int):
    _check(lib().pdv_cancel(C.c_void_p(ctx), C.c_uint64(ticket)))


def pdv_debug_get(ctx: int, reset: bool = False) -> dict:
    """The debug build's failed-check record (debug_build 0 in the release
    library), optionally cleared."""
    d = pdv_debug_info()
    _check(lib().pdv_debug_get(C.c_void_p(ctx), C.byref(d), int(bool(reset))))
    out = {f: getattr(d, f) for f, _ in pdv_debug_info._fields_}
    out["site_name"] = DEBUG_SITES[out["site"]] if out["site"] < len(DEBUG_SITES) else out["site"]
    return out


def pdv_debug_set_trace(ctx: int, n_trace: int, max_vertices: int, out=None):
    """Arm a path trace of the next spectrum call with per-packet records;
    ``out``: TRACE_DTYPE array [n_trace, max_vertices] that must stay alive
    until that call returns (n_trace = 0 disarms)."""
    _check(lib().pdv_debug_set_trace(C.c_void_p(ctx), int(n_trace), int(max_vertices),
                                     C.c_void_p(out.ctypes.data) if out is not None else None))


def _addr(a):
    """(address, on_device) of a contiguous numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.is_cuda
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, False


def pdv_ss_spectrum(ctx: int, sets, n_sets: int, n_bins: int, v_lo: float, v_hi: float,
                    out, per_dv: bool = False):
    """Single-scattering spectra (Eq. 28) of ``n_sets`` parameter sets integrated
    over ``n_bins`` bins. ``sets``: SS_SET_DTYPE array, or a CUDA tensor of
    float64 [n_sets, 5] (beta, tau0, v_fs, v_max, prefactor); ``out``: float64
    [n_sets * n_bins] numpy array or CUDA tensor."""
    ps, dev_in = _addr(sets)
    po, dev_out = _addr(out)
    flags = (PDV_IN_DEVICE if dev_in else 0) | (PDV_OUT_DEVICE if dev_out else 0) | \
        (PDV_PER_DV if per_dv else 0)
    _check(lib().pdv_ss_spectrum(C.c_void_p(ctx), C.c_void_p(ps), n_sets, n_bins, v_lo, v_hi,
                                 flags, C.c_void_p(po)))


def pdv_extract_peaks(ctx: int, spectra, n_spectra: int, n_bins: int, v_lo: float, v_hi: float,
                      v_fs: float, k_c: int, x_min: float, x_max: float, out,
                      simt: bool = False):
    """Main-peak extraction (Eq. 29-35). ``spectra``: float64 [n_spectra, n_bins]
    (numpy or CUDA tensor); ``out``: PEAK_DTYPE array, or a CUDA uint8 tensor of
    n_spectra * 48 bytes. ``simt``: both products as FP32 FMAs on the CUDA
    cores (PDV_EXTRACT_SIMT) instead of the tensor cores."""
    ps, dev_in = _addr(spectra)
    po, dev_out = _addr(out)
    flags = (PDV_IN_DEVICE if dev_in else 0) | (PDV_OUT_DEVICE if dev_out else 0) | \
        (PDV_EXTRACT_SIMT if simt else 0)
    o = pdv_peak_opts(k_c=k_c, reserved=0, x_min=x_min, x_max=x_max)
    _check(lib().pdv_extract_peaks(C.c_void_p(ctx), C.c_void_p(ps), n_spectra, n_bins, v_lo,
                                   v_hi, v_fs, C.byref(o), flags, C.c_void_p(po)))


# ------------------------------------------------------------------ conveniences
def ss_spectrum(ctx: "Context", params, n_bins: int, v_lo: float, v_hi: float,
                per_dv: bool = False) -> np.ndarray:
    """Host convenience: ``params`` is a sequence of dicts or tuples (beta,
    tau0, v_fs, v_max, prefactor); returns float64 [n_sets, n_bins]."""
    arr = np.zeros(len(params), dtype=SS_SET_DTYPE)
    for i, p in enumerate(params):
        if isinstance(p, dict):
            p = (p["beta"], p["tau0"], p["v_fs"], p.get("v_max", 0.0), p.get("prefactor", 1.0))
        p = tuple(p)
        if not 3 <= len(p) <= 5:
            raise ValueError("a set is (beta, tau0, v_fs[, v_max[, prefactor]])")
        arr[i] = p + (0.0, 1.0)[len(p) - 3:]       # defaults: untruncated, unit prefactor
    out = np.zeros(len(params) * n_bins)
    pdv_ss_spectrum(ctx.handle, arr, len(params), n_bins, v_lo, v_hi, out, per_dv)
    return out.reshape(len(params), n_bins)


def extract_peaks(ctx: "Context", spectra, v_lo: float, v_hi: float, v_fs: float, k_c: int,
                  x_min: float = -math.inf, x_max: float = math.inf,
                  simt: bool = False) -> np.ndarray:
    """Host convenience: spectra float64 [n_spectra, n_bins] -> PEAK_DTYPE array."""
    s = np.ascontiguousarray(spectra, dtype=np.float64)
    if s.ndim == 1:
        s = s[None, :]
    out = np.zeros(s.shape[0], dtype=PEAK_DTYPE)
    pdv_extract_peaks(ctx.handle, s, s.shape[0], s.shape[1], v_lo, v_hi, v_fs, k_c, x_min, x_max,
                      out, simt)
    return out


class Context:
    """A libpdv context on one device (``stream``: a cudaStream_t as int)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None,
                 allocator: Optional[pdv_allocator] = None):
        self.allocator = allocator          # its callbacks must outlive the context
        self.handle = pdv_ctx_create(device, stream, allocator)

    def close(self):
        if self.handle:
            pdv_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        return pdv_get_stats(self.handle)

    def set_tuning(self, **kw):
        pdv_set_tuning(self.handle, **kw)

    def mie_table(self, m, wavelength_nm, d_median_um, sigma_ln, n_size=256, n_angle=1801):
        return pdv_mie_table(self.handle, m, wavelength_nm, d_median_um, sigma_ln, n_size, n_angle)


def phase_table(ctx: Context, wl):
    """(theta, p, q_ext, albedo) for a workload, computed by the library."""
    ph = wl.phase
    if ph.kind == "hg":
        th, p = pdv_phase_hg(ph.g, ph.n_angle)
        return th, p, ph.q_ext, ph.albedo
    if ph.kind == "mie":
        th, p, q_ext, albedo, _ = ctx.mie_table(ph.m, wl.wavelength * 1e9, wl.d_m * 1e6,
                                                wl.sigma_ln, ph.n_size, ph.n_angle)
        return th, p, q_ext, albedo
    if ph.kind == "table":
        return np.asarray(ph.theta, np.float64), np.asarray(ph.p, np.float64), ph.q_ext, ph.albedo
    if ph.kind == "mie_iso":
        # uniform scattering with the cloud's size-averaged Mie extinction and albedo
        th, _, q_ext, albedo, _ = ctx.mie_table(ph.m, wl.wavelength * 1e9, wl.d_m * 1e6,
                                                wl.sigma_ln, ph.n_size, ph.n_angle)
        return th, np.ones_like(th), q_ext, albedo
    raise ValueError(ph.kind)


class Cloud:
    """Device-resident cloud + phase table built from a workload."""

    def __init__(self, ctx: Context, wl, table=None, table_nodes: int = 0):
        self.ctx = ctx
        d = pdv_cloud_desc()
        d.rho_kg_m3 = wl.rho
        d.area_mass_mg_cm2 = wl.m0 / 1e-2
        d.v_fs = wl.v_fs
        d.reflectivity = wl.reflectivity
        d.surface_mode = wl.surface_mode
        d.profile_kind = 0 if wl.profile_kind == "exponential" else 1
        d.beta = wl.beta
        d.v_max = wl.v_max
        self._pv = self._pf = None
        if d.profile_kind == 1:
            self._pv = np.ascontiguousarray(wl.prof_v, np.float64)
            self._pf = np.ascontiguousarray(wl.prof_f, np.float64)
            d.prof_v = _dp(self._pv)
            d.prof_dmdv = _dp(self._pf)
            d.prof_n = len(self._pv)
        d.d_median_um = wl.d_m * 1e6
        d.sigma_ln = wl.sigma_ln
        d.wavelength_nm = wl.wavelength * 1e9
        d.table_nodes = table_nodes
        self.handle = pdv_create_cloud(ctx.handle, d)
        th, p, q_ext, albedo = table if table is not None else phase_table(ctx, wl)
        pdv_set_phase_table(self.handle, th, p, q_ext, albedo)
        self.table = (th, p, q_ext, albedo)

    def info(self) -> dict:
        return pdv_cloud_get_info(self.handle)

    def close(self):
        if self.handle:
            pdv_destroy_cloud(self.handle)
            self.handle = None


class Request:
    """A pdv_request plus the host arrays it points to (kept alive here)."""

    def __init__(self, cloud: Cloud, wl, precision=None, n_packets=None, packet_begin=0,
                 raw=True, counters=True, packets=False, per_dv=False, device_out=None,
                 snapshots=None):
        r = pdv_request()
        r.cloud = cloud.handle
        r.probe = pdv_probe(wl.z_probe * 1e3, wl.r_beam * 1e3, wl.r_ap * 1e3, wl.cone_alpha)
        t = wl.t_snap if snapshots is None else snapshots
        self.t_us = np.ascontiguousarray(np.asarray(t, np.float64) * 1e6)
        r.t_snap_us = _dp(self.t_us)
        r.n_snap = len(self.t_us)
        r.n_packets = int(wl.n_packets if n_packets is None else n_packets)
        r.packet_begin = int(packet_begin)
        r.seed = int(wl.seed)
        r.stream_id = int(wl.stream_id)
        r.max_events = int(wl.max_events)
        r.n_layers = int(getattr(wl, "n_layers", 0))
        r.n_bins = int(wl.n_bins)
        r.v_lo = wl.v_lo
        r.v_hi = wl.v_hi
        prec = precision or wl.precision
        r.precision = PDV_PREC_FP64 if prec in ("fp64", PDV_PREC_FP64) else PDV_PREC_FP32
        r.flags = PDV_PER_DV if per_dv else 0
        if getattr(wl, "implicit_capture", False):
            r.flags |= PDV_IMPLICIT_CAPTURE
        if getattr(wl, "horizontal_launch", False):
            r.flags |= PDV_TEST_HORIZONTAL_LAUNCH
        ns, nb = r.n_snap, r.n_bins
        self.device_out = device_out
        if device_out is not None:
            # caller-provided device tensors (e.g. torch CUDA tensors): data_ptr()
            r.flags |= PDV_OUT_DEVICE
            r.out_spectrum = device_out["spectrum"].data_ptr()
            r.out_raw = device_out["raw"].data_ptr() if "raw" in device_out else None
            r.out_counters = device_out["counters"].data_ptr() if "counters" in device_out else None
            r.out_packets = device_out["packets"].data_ptr() if "packets" in device_out else None
            self.spectrum = self.raw = self.counters = self.packets = None
        else:
            self.spectrum = np.zeros((ns, nb), np.float64)
            self.raw = np.zeros((ns, nb + 2), np.uint64) if raw else None
            self.counters = (pdv_counters * ns)() if counters else None
            self.packets = np.zeros(r.n_packets, PACKET_DTYPE) if packets else None
            r.out_spectrum = self.spectrum.ctypes.data
            r.out_raw = self.raw.ctypes.data if raw else None
            r.out_counters = C.addressof(self.counters) if counters else None
            r.out_packets = self.packets.ctypes.data if packets else None
        self.c = r

    def result(self) -> dict:
        out = {"spectrum": self.spectrum}
        if self.raw is not None:
            out["raw"] = self.raw
            out["hist"] = self.raw[:, 1:-1]
        if self.counters is not None:
            out["counters"] = np.array([[getattr(c, n) for n in COUNTER_NAMES]
                                        for c in self.counters], np.uint64)
        if self.packets is not None:
            out["packets"] = self.packets
        return out


def simulate_spectrum(ctx: Context, cloud: Cloud, wl, trace=None, debug_check=False,
                      **kw) -> dict:
    """One spectrum request. Debug build only: ``trace=(n, max_vertices)``
    also returns the paths of the first n packets (``out["trace"]``,
    TRACE_DTYPE [n, max_vertices]; needs ``packets=True``), and
    ``debug_check`` sets PDV_TEST_DEBUG_CHECK."""
    req = Request(cloud, wl, **kw)
    if debug_check:
        req.c.flags |= PDV_TEST_DEBUG_CHECK
    tr = None
    if trace is not None:
        tr = np.zeros(tuple(trace), TRACE_DTYPE)
        pdv_debug_set_trace(ctx.handle, trace[0], trace[1], tr)
    try:
        pdv_simulate_spectrum(ctx.handle, req.c)
    finally:
        if tr is not None:
            pdv_debug_set_trace(ctx.handle, 0, 0)
    out = req.result()
    if tr is not None:
        out["trace"] = tr
    return out


def simulate_batch(ctx: Context, clouds: Sequence[Cloud], wls, **kw) -> list:
    reqs = [Request(c, w, **kw) for c, w in zip(clouds, wls)]
    pdv_simulate_batch(ctx.handle, [r.c for r in reqs])
    return [r.result() for r in reqs]


def counters_dict(row) -> dict:
    return {k: int(v) for k, v in zip(COUNTER_NAMES, row)}


def cuda_stream_handle(torch_stream=None) -> int:
    """The cudaStream_t of a torch stream (torch is used only as plumbing)."""
    import torch
    s = torch_stream or torch.cuda.current_stream()
    return int(s.cuda_stream)
