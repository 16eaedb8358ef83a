"""Python access to the FP64 CPU oracle (``pdv_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg use this module. It never imports the
product package; a workload is read by attribute (duck typing), in SI units.

The oracle follows the Monte Carlo of Shi et al., arXiv:2012.00963, Section II:
Beer–Lambert free paths (Eq. 7, Eq. 10), scatter/absorb branch (Eq. 11), Mie
phase function (Eq. 12-14), azimuth (Eq. 15), rotation (Eq. 16-17), Doppler
update (Eq. 4, Eq. 18), diffuse free-surface reflection, tally (Eq. 19).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NCOUNTERS = 16
NORDER = 5
COUNTER_NAMES = [
    "launched", "events", "scatters", "surface_hits", "escapes", "detected",
    "w_detected", "w_under", "w_over", "w_escaped_undetected", "w_absorbed_particle",
    "w_absorbed_surface", "w_truncated", "truncated", "w_roulette_dropped", "w_roulette_gained",
]
FATE_ESCAPED, FATE_ABS_PARTICLE, FATE_ABS_SURFACE, FATE_TRUNCATED, FATE_DROPPED = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pdv_oracle.h"))):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
            "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("m0", C.c_double), ("v_fs", C.c_double),
        ("reflectivity", C.c_double), ("surface_mode", C.c_int), ("profile_kind", C.c_int),
        ("beta", C.c_double), ("v_max", C.c_double),
        ("prof_v", C.POINTER(C.c_double)), ("prof_f", C.POINTER(C.c_double)),
        ("prof_n", C.c_int),
        ("d_m", C.c_double), ("sigma_ln", C.c_double), ("q_ext", C.c_double),
        ("albedo", C.c_double),
        ("n_phase", C.c_int), ("theta", C.POINTER(C.c_double)), ("p", C.POINTER(C.c_double)),
        ("z_probe", C.c_double), ("r_beam", C.c_double), ("r_ap", C.c_double),
        ("cone_alpha", C.c_double),
        ("n_snap", C.c_int), ("t_snap", C.POINTER(C.c_double)),
        ("n_bins", C.c_int), ("v_lo", C.c_double), ("v_hi", C.c_double),
        ("packet_begin", C.c_uint64), ("n_packets", C.c_uint64), ("seed", C.c_uint64),
        ("stream_id", C.c_uint32), ("max_events", C.c_uint32), ("n_layers", C.c_uint32),
        ("implicit_capture", C.c_uint32), ("test_horizontal_launch", C.c_uint32),
        ("spread_runs", C.c_uint32),
        ("spread_flight", C.c_double), ("spread_turn", C.c_double), ("spread_store", C.c_double),
    ]


PACKET_DTYPE = np.dtype([
    ("n_events", np.uint32), ("n_scatters", np.uint32), ("n_surface", np.uint32),
    ("fate", np.uint32), ("weight", np.uint64), ("v_app", np.float64),
    ("detect_mask", np.uint64), ("v_app_spread", np.float64), ("n_unstable", np.uint32),
    ("_pad", np.uint32),
])

# Rounding sensitivity of v_app (packet records only): perturbed FP64 re-runs
# with random errors of the size of a binary32 walk's roundings, as standard
# deviations in units of u = 2^-24: a flight's optical length (logarithm and two
# products, relative), each new direction component (polar angle, sin/cos,
# rotation and renormalisation, absolute), and the storage of each component
# (relative). Derived in DESIGN from the FP32 kernel's operations.
SPREAD_RUNS = 8
SPREAD_SD = (2.0, 3.0, 1.0)
VERTEX_DTYPE = np.dtype([
    ("x", np.float64), ("y", np.float64), ("z", np.float64), ("v", np.float64),
    ("ux", np.float64), ("uy", np.float64), ("uz", np.float64), ("kind", np.int32),
    ("_pad", np.int32),
])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            u64p = C.POINTER(C.c_uint64)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_cloud_constants.argtypes = [C.POINTER(_Problem), dp, dp, dp, dp]
            L.orc_cloud_constants.restype = C.c_int
            L.orc_profile_cdf.argtypes = [C.POINTER(_Problem), C.c_double]
            L.orc_profile_cdf.restype = C.c_double
            L.orc_profile_inverse.argtypes = [C.POINTER(_Problem), C.c_double]
            L.orc_profile_inverse.restype = C.c_double
            L.orc_mie_single.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, dp,
                                         dp, dp]
            L.orc_mie_single.restype = C.c_int
            L.orc_mie_table.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.orc_mie_table.restype = C.c_int
            L.orc_hg_table.argtypes = [C.c_double, C.c_int, dp, dp]
            L.orc_hg_table.restype = None
            L.orc_phase_cdf.argtypes = [C.c_int, dp, dp, u32p, dp]
            L.orc_phase_cdf.restype = C.c_int
            L.orc_phase_sample.argtypes = [C.c_int, dp, u32p, C.c_uint32]
            L.orc_phase_sample.restype = C.c_double
            L.orc_rotate.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_rotate.restype = None
            L.orc_phase_ar_cos.argtypes = [C.POINTER(_Problem), C.c_uint64, C.c_uint32]
            L.orc_phase_ar_cos.restype = C.c_double
            L.orc_simulate.argtypes = [C.POINTER(_Problem), C.c_int, u64p, u64p, u64p, C.c_void_p,
                                       C.c_int, C.c_int, C.c_void_p]
            L.orc_simulate.restype = C.c_int
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u32ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _u64ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_u32ptr(c), _u32ptr(k), _u32ptr(out))
    return out


def mie_single(x, m, mu=None):
    """(Q_ext, Q_sca, Q_back, g), |S1|^2, |S2|^2 at mu, S(0), n_terms."""
    mu = np.zeros(0) if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
    s11 = np.zeros(len(mu))
    s22 = np.zeros(len(mu))
    q = np.zeros(4)
    s0 = np.zeros(2)
    n = lib().orc_mie_single(float(x), float(np.real(m)), float(np.imag(m)), len(mu), _dptr(mu),
                             _dptr(s11), _dptr(s22), _dptr(q), _dptr(s0))
    return q, s11, s22, complex(s0[0], s0[1]), n


def mie_table(m, wavelength, d_m, sigma_ln, n_angle=1801, n_size=256):
    theta = np.zeros(n_angle)
    p = np.zeros(n_angle)
    q = np.zeros(3)
    rc = lib().orc_mie_table(float(np.real(m)), float(np.imag(m)), float(wavelength), float(d_m),
                             float(sigma_ln), int(n_size), int(n_angle), _dptr(theta), _dptr(p),
                             _dptr(q[0:1]), _dptr(q[1:2]), _dptr(q[2:3]))
    if rc != 0:
        raise ValueError("orc_mie_table: invalid input")
    return theta, p, float(q[0]), float(q[1]), float(q[2])


def hg_table(g, n=1801):
    theta = np.zeros(n)
    p = np.zeros(n)
    lib().orc_hg_table(float(g), int(n), _dptr(theta), _dptr(p))
    return theta, p


def phase_cdf(theta, p):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    cq = np.zeros(len(theta), np.uint32)
    g = np.zeros(1)
    rc = lib().orc_phase_cdf(len(theta), _dptr(theta), _dptr(p), _u32ptr(cq), _dptr(g))
    if rc != 0:
        raise ValueError("orc_phase_cdf: invalid table")
    return cq, float(g[0])


def phase_sample(theta, cq, m):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    cq = np.ascontiguousarray(cq, dtype=np.uint32)
    return lib().orc_phase_sample(len(theta), _dptr(theta), _u32ptr(cq), int(m))


def rotate(u, cos_t, sin_t, cos_p, sin_p):
    v = np.ascontiguousarray(u, dtype=np.float64).copy()
    lib().orc_rotate(_dptr(v), cos_t, sin_t, cos_p, sin_p)
    return v


def phase_ar_cos(wl, packets, step=1, table=None):
    """cos(theta) from the layer-stepping scheme's acceptance-rejection for each
    packet index in `packets` at the given step (seed, stream and phase table
    of the workload)."""
    prob = Problem(wl, table=table)
    return np.array([lib().orc_phase_ar_cos(C.byref(prob.pb), int(k), int(step))
                     for k in packets])


# ---------------------------------------------------------------- problems
def phase_table(wl):
    """The oracle's own phase table, albedo and Q_ext for a workload."""
    ph = wl.phase
    if ph.kind == "hg":
        theta, p = hg_table(ph.g, ph.n_angle)
        return theta, p, ph.q_ext, ph.albedo
    if ph.kind == "mie":
        theta, p, q_ext, albedo, _ = mie_table(ph.m, wl.wavelength, wl.d_m, wl.sigma_ln,
                                               ph.n_angle, ph.n_size)
        return theta, p, q_ext, albedo
    if ph.kind == "table":
        return (np.asarray(ph.theta, np.float64), np.asarray(ph.p, np.float64), ph.q_ext,
                ph.albedo)
    if ph.kind == "mie_iso":
        # uniform scattering (Section II.D, second case of Fig. 6): the size-averaged
        # Mie extinction and albedo of the cloud, with an isotropic phase function
        theta, _, q_ext, albedo, _ = mie_table(ph.m, wl.wavelength, wl.d_m, wl.sigma_ln,
                                               ph.n_angle, ph.n_size)
        return theta, np.ones_like(theta), q_ext, albedo
    raise ValueError(ph.kind)


class Problem:
    """Holds an ``orc_problem`` and the arrays it points to."""

    def __init__(self, wl, n_packets=None, packet_begin=0, snapshots=None, table=None):
        theta, p, q_ext, albedo = table if table is not None else phase_table(wl)
        self.theta = np.ascontiguousarray(theta, np.float64)
        self.p = np.ascontiguousarray(p, np.float64)
        t = wl.t_snap if snapshots is None else snapshots
        self.t_snap = np.ascontiguousarray(t, np.float64)
        pb = _Problem()
        pb.rho = wl.rho
        pb.m0 = wl.m0
        pb.v_fs = wl.v_fs
        pb.reflectivity = wl.reflectivity
        pb.surface_mode = wl.surface_mode
        pb.profile_kind = 0 if wl.profile_kind == "exponential" else 1
        pb.beta = wl.beta
        pb.v_max = wl.v_max
        if pb.profile_kind == 1:
            self.prof_v = np.ascontiguousarray(wl.prof_v, np.float64)
            self.prof_f = np.ascontiguousarray(wl.prof_f, np.float64)
            pb.prof_v = _dptr(self.prof_v)
            pb.prof_f = _dptr(self.prof_f)
            pb.prof_n = len(self.prof_v)
        pb.d_m = wl.d_m
        pb.sigma_ln = wl.sigma_ln
        pb.q_ext = q_ext
        pb.albedo = albedo
        pb.n_phase = len(self.theta)
        pb.theta = _dptr(self.theta)
        pb.p = _dptr(self.p)
        pb.z_probe = wl.z_probe
        pb.r_beam = wl.r_beam
        pb.r_ap = wl.r_ap
        pb.cone_alpha = wl.cone_alpha
        pb.n_snap = len(self.t_snap)
        pb.t_snap = _dptr(self.t_snap)
        pb.n_bins = wl.n_bins
        pb.v_lo = wl.v_lo
        pb.v_hi = wl.v_hi
        pb.packet_begin = packet_begin
        pb.n_packets = wl.n_packets if n_packets is None else n_packets
        pb.seed = wl.seed
        pb.stream_id = wl.stream_id
        pb.max_events = wl.max_events
        pb.n_layers = getattr(wl, "n_layers", 0)
        pb.implicit_capture = int(bool(getattr(wl, "implicit_capture", False)))
        pb.test_horizontal_launch = int(bool(getattr(wl, "horizontal_launch", False)))
        pb.spread_runs = 0
        pb.spread_flight, pb.spread_turn, pb.spread_store = SPREAD_SD
        self.pb = pb
        self.q_ext = q_ext
        self.albedo = albedo

    def constants(self):
        tau, vb, vt, ds = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        rc = lib().orc_cloud_constants(C.byref(self.pb), C.byref(tau), C.byref(vb), C.byref(vt),
                                       C.byref(ds))
        if rc != 0:
            raise ValueError("invalid cloud")
        return dict(tau_tot=tau.value, v_bot=vb.value, v_top=vt.value, d_sauter=ds.value)

    def cdf(self, v):
        return lib().orc_profile_cdf(C.byref(self.pb), float(v))

    def inverse(self, s):
        return lib().orc_profile_inverse(C.byref(self.pb), float(s))


def simulate(wl, n_threads=None, n_packets=None, packet_begin=0, snapshots=None, order=False,
             packets=False, n_trace=0, max_vertices=64, table=None, spread_runs=None,
             spread_sd=None):
    """Run the oracle. Returns a dict with ``hist`` [n_snap, n_bins] (uint64, 2^32
    weight units), ``counters`` [n_snap, NCOUNTERS], optionally ``order``
    [n_snap, NORDER, n_bins], ``packets`` (PACKET_DTYPE) and ``trace``. With
    packet records, ``spread_runs`` perturbed re-runs (default SPREAD_RUNS)
    give each packet's ``v_app_spread``; ``spread_sd`` overrides SPREAD_SD."""
    pr = Problem(wl, n_packets=n_packets, packet_begin=packet_begin, snapshots=snapshots,
                 table=table)
    pb = pr.pb
    if packets:
        pb.spread_runs = SPREAD_RUNS if spread_runs is None else int(spread_runs)
        if spread_sd is not None:
            pb.spread_flight, pb.spread_turn, pb.spread_store = spread_sd
    ns, nb = pb.n_snap, pb.n_bins
    hist = np.zeros((ns, nb), np.uint64)
    cnt = np.zeros((ns, NCOUNTERS), np.uint64)
    oh = np.zeros((ns, NORDER, nb), np.uint64) if order else None
    pk = np.zeros(pb.n_packets, PACKET_DTYPE) if packets else None
    tr = np.zeros((n_trace, max_vertices), VERTEX_DTYPE) if n_trace else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = lib().orc_simulate(
        C.byref(pb), int(n_threads), _u64ptr(hist), _u64ptr(cnt),
        _u64ptr(oh) if oh is not None else None,
        pk.ctypes.data if pk is not None else None, int(n_trace), int(max_vertices),
        tr.ctypes.data if tr is not None else None)
    if rc != 0:
        raise ValueError("orc_simulate: invalid problem")
    out = dict(hist=hist, counters=cnt, q_ext=pr.q_ext, albedo=pr.albedo, **pr.constants())
    if oh is not None:
        out["order"] = oh
    if pk is not None:
        out["packets"] = pk
    if tr is not None:
        out["trace"] = tr
    return out


def counters_dict(row):
    return {k: int(v) for k, v in zip(COUNTER_NAMES, row)}
