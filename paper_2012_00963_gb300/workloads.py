"""Seeded synthetic workloads for the PDV Monte Carlo (shared input generators).

This module only describes inputs: cloud, phase-function choice, probe, snapshot
times and packet counts, in SI units, plus the seeded draws of the batched and
served workloads. It holds none of the method's arithmetic, so that the CUDA
path and the FP64 oracle can both be fed from it without sharing code.

The named workloads follow the paper's synthetic Sn clouds (Section II.D and
Section III.A: exponential velocity law Eq. 20, log-normal sizes Eq. 21,
lambda = 1550 nm, vacuum, z = v t) at the sizes of the benchmark set:

* ``cfg1`` — monodisperse 2 um, 0.5 mg/cm^2 (tau ~ 1 with Q_ext = 2), beta = 5
  on [2000, 6000] m/s, HG g = 0.7 and albedo 0.6 on 1801 angles, one snapshot
  at 1 us, 1e6 packets, 200 bins over 0-6000 m/s.
* ``cfg2`` — log-normal d_m = 3 um, sigma = 0.5, Mie m = 3 + 9i, 5 mg/cm^2,
  beta = 5, 50 snapshots 0.5-5 us, 1e8 packets per snapshot, 600 bins 0-8000.
* ``cfg3`` — heavy multiple scattering: monodisperse 1 um, 20 mg/cm^2, beta = 3,
  Mie m = 3 + 9i; FP32 and FP64 GPU paths against the oracle.
* ``cfg4`` — 256 parameter sets drawn from a seed (batched launch).
* ``cfg5`` — Poisson request stream for the serving loop.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

MG_CM2 = 1.0e-2          # 1 mg/cm^2 in kg/m^2
UM = 1.0e-6
NM = 1.0e-9
MM = 1.0e-3
US = 1.0e-6


@dataclass
class Phase:
    """Phase-function choice: Henyey–Greenstein with given albedo and Q_ext,
    size-averaged Mie for a complex index, isotropic scattering with the Mie
    extinction and albedo ("mie_iso"), or an explicit table."""
    kind: str = "hg"                  # "hg" | "mie" | "mie_iso" | "table"
    g: float = 0.7
    albedo: float = 0.6
    q_ext: float = 2.0
    m: complex = 3.0 + 9.0j
    n_angle: int = 1801
    n_size: int = 256
    theta: Optional[Sequence[float]] = None
    p: Optional[Sequence[float]] = None


@dataclass
class Workload:
    # cloud (SI)
    rho: float = 7290.0
    m0: float = 0.5 * MG_CM2
    v_fs: float = 2000.0
    reflectivity: float = 0.6
    surface_mode: int = 0             # 0 uniform polar angle, 1 Lambertian, 2 specular
    profile_kind: str = "exponential"  # or "tabulated"
    beta: float = 5.0
    v_max: float = 6000.0             # 0 -> mass-tail rule
    prof_v: Optional[Sequence[float]] = None
    prof_f: Optional[Sequence[float]] = None
    d_m: float = 2.0 * UM
    sigma_ln: float = 0.0
    wavelength: float = 1550.0 * NM
    phase: Phase = field(default_factory=Phase)
    # probe
    z_probe: float = 50.0 * MM
    r_beam: float = 0.5 * MM
    r_ap: float = 1.0 * MM            # <= 0: unlimited
    cone_alpha: float = 0.1           # >= pi/2: all upward
    # snapshots and tally
    t_snap: Sequence[float] = (1.0 * US,)
    n_bins: int = 200
    v_lo: float = 0.0
    v_hi: float = 6000.0
    # packets
    n_packets: int = 1_000_000
    seed: int = 1
    stream_id: int = 0
    max_events: int = 1_000_000       # with layer stepping: the step limit
    n_layers: int = 0                 # 0 exact free paths; > 0 the paper's H / n_layers steps
    implicit_capture: bool = False    # weight omega per interaction + Russian roulette (exact paths)
    horizontal_launch: bool = False   # test hook: packets start along +x (the |u_z| < 1e-9 rule)
    precision: str = "fp32"           # "fp32" | "fp64"
    name: str = "custom"

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def cfg1(**kw) -> Workload:
    """Plain FP64-accurate transport case (tin, monodisperse 2 um, HG)."""
    return Workload(name="cfg1").replace(**kw)


def cfg2(**kw) -> Workload:
    """Log-normal 3 um / 0.5, Mie 3+9i at 1550 nm, 5 mg/cm^2, 50 snapshots."""
    wl = Workload(
        name="cfg2", m0=5.0 * MG_CM2, beta=5.0, v_max=0.0, d_m=3.0 * UM, sigma_ln=0.5,
        phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=256),
        t_snap=tuple(np.linspace(0.5, 5.0, 50) * US), n_bins=600, v_lo=0.0, v_hi=8000.0,
        n_packets=100_000_000, seed=2)
    return wl.replace(**kw)


def cfg3(**kw) -> Workload:
    """Heavy multiple scattering: 20 mg/cm^2, monodisperse 1 um, beta = 3."""
    wl = Workload(
        name="cfg3", m0=20.0 * MG_CM2, beta=3.0, v_max=0.0, d_m=1.0 * UM, sigma_ln=0.0,
        phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=1),
        t_snap=(1.0 * US,), n_bins=600, v_lo=0.0, v_hi=8000.0, n_packets=1_000_000_000,
        seed=3)
    return wl.replace(**kw)


def cfg4_sets(n_sets: int = 256, seed: int = 4, n_min: float = 1e5, n_max: float = 1e8,
              n_bins: int = 400) -> List[Workload]:
    """256 parameter sets: beta ~ U(2, 10), m0 ~ logU(0.1, 20) mg/cm^2,
    d ~ logU(0.5, 10) um, v_fs ~ U(1.5, 3) km/s, t ~ U(1, 4) us, packets ~
    logU(n_min, n_max); monodisperse Mie 3+9i, one snapshot, bins over
    [0, v_max of the set]. The probe sits 120 mm above the sample: the fastest
    clouds of these ranges (beta = 2, v_fs = 3 km/s) reach about 95 mm at 4 us."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_sets):
        beta = float(rng.uniform(2.0, 10.0))
        m0 = float(np.exp(rng.uniform(np.log(0.1), np.log(20.0)))) * MG_CM2
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(10.0)))) * UM
        v_fs = float(rng.uniform(1500.0, 3000.0))
        t = float(rng.uniform(1.0, 4.0)) * US
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        v_top = v_fs * (1.0 + math.log(1.0e6) / beta)   # mass-tail rule of the cloud
        out.append(Workload(
            name="cfg4[%d]" % i, m0=m0, beta=beta, v_max=0.0, v_fs=v_fs, d_m=d, sigma_ln=0.0,
            phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=1), t_snap=(t,),
            n_bins=n_bins, v_lo=0.0, v_hi=v_top, n_packets=n, seed=1000 + i, stream_id=i,
            z_probe=120.0 * MM))
    return out


@dataclass
class Arrival:
    t: float              # arrival time, s
    beta: float
    m0: float             # kg/m^2
    d_m: float            # m
    n_packets: int
    seed: int


def cfg5_arrivals(rate: float = 200.0, duration: float = 60.0, seed: int = 5,
                  n_min: float = 1e5, n_max: float = 1e7) -> List[Arrival]:
    """Poisson request stream (rate per second over ``duration`` seconds) of
    candidate (beta, m0, d) sets around a sweep, packets ~ logU(n_min, n_max)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        out.append(Arrival(
            t=t, beta=float(rng.uniform(3.0, 10.0)),
            m0=float(np.exp(rng.uniform(np.log(1.0), np.log(10.0)))) * MG_CM2,
            d_m=float(np.exp(rng.uniform(np.log(1.0), np.log(4.0)))) * UM,
            n_packets=int(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))),
            seed=50_000 + i))
        i += 1
    return out


def cfg5_request(a: Arrival, **kw) -> Workload:
    """Spectrum request of the serving stream for one arrival (HG phase so that
    no per-request Mie table is needed; beams and probe as in cfg1)."""
    wl = Workload(name="cfg5", m0=a.m0, beta=a.beta, v_max=0.0, d_m=a.d_m,
                  phase=Phase(kind="hg", g=0.7, albedo=0.6, q_ext=2.0), n_bins=400,
                  v_lo=0.0, v_hi=8000.0, n_packets=a.n_packets, seed=a.seed)
    return wl.replace(**kw)


def model_sets(n_sets: int = 100_000, seed: int = 6, v_fs: float = 2000.0) -> np.ndarray:
    """Parameter sets of the single-scattering model (Section III.B): beta ~
    U(2, 12), tau0 ~ logU(2, 60) (the paper's cases run from tau0 = 8.6 to
    28.8), one free-surface velocity for the batch (a spectrogram of one
    shot), untruncated law, unit prefactor. Columns: beta, tau0, v_fs, v_max
    (0: untruncated), prefactor."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n_sets, 5), dtype=np.float64)
    out[:, 0] = rng.uniform(2.0, 12.0, n_sets)
    out[:, 1] = np.exp(rng.uniform(np.log(2.0), np.log(60.0), n_sets))
    out[:, 2] = v_fs
    out[:, 4] = 1.0
    return out


def spectrum_noise(shape, seed: int = 7, level: float = 0.02) -> np.ndarray:
    """Multiplicative noise factors 1 + level * N(0, 1) for synthetic measured
    spectra (seeded)."""
    return 1.0 + level * np.random.default_rng(seed).standard_normal(shape)


def fig6(case: int = 1, **kw) -> Workload:
    """The comparison cloud of Section II.D (Fig. 6): tin, m0 = 10.7 mg/cm^2,
    log-normal d_m = 1.5 um, sigma = 0.5, beta = 8, lambda = 1550 nm; case 1
    scatters by the Mie phase function, case 2 isotropically (with the same
    Mie extinction and albedo). Every upward photon is counted, as the paper
    does; 600 bins over 0-8000 m/s, one snapshot at 1 us, 1e7 packets."""
    if case not in (1, 2):
        raise ValueError("case 1 (Mie) or 2 (uniform scattering)")
    wl = Workload(
        name="fig6-case%d" % case, m0=10.7 * MG_CM2, beta=8.0, v_max=0.0, d_m=1.5 * UM,
        sigma_ln=0.5, phase=Phase(kind="mie" if case == 1 else "mie_iso", m=3.0 + 9.0j,
                                  n_angle=1801, n_size=256),
        r_ap=0.0, cone_alpha=math.pi / 2, t_snap=(1.0 * US,), n_bins=600, v_lo=0.0,
        v_hi=8000.0, n_packets=10_000_000, seed=8)
    return wl.replace(**kw)


# The two clouds of Figs. 13-15 (Section III.B), quoted there with the
# single-scattering optical thickness tau0 of Eq. 27.
FIG13_CLOUDS = (
    dict(label="tau0=23.4", tau0_paper=23.4, m0=20.0 * MG_CM2, d_m=1.5 * UM, sigma_ln=0.5),
    dict(label="tau0=8.6", tau0_paper=8.6, m0=10.0 * MG_CM2, d_m=2.0 * UM, sigma_ln=0.5),
)


def fig13(cloud: int, beta: float, **kw) -> Workload:
    """One Monte Carlo case of the peak-position / curvature study of
    Figs. 13-15: cloud 0 (tau0 = 23.4) or 1 (tau0 = 8.6) at velocity
    coefficient beta; Mie 3+9i at 1550 nm, every upward photon counted, 1200
    bins over 0-8000 m/s, 1e7 packets (the paper's count)."""
    c = FIG13_CLOUDS[cloud]
    wl = Workload(
        name="fig13-%s-beta%g" % (c["label"], beta), m0=c["m0"], beta=beta, v_max=0.0,
        d_m=c["d_m"], sigma_ln=c["sigma_ln"],
        phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=256),
        r_ap=0.0, cone_alpha=math.pi / 2, t_snap=(1.0 * US,), n_bins=1200, v_lo=0.0,
        v_hi=8000.0, n_packets=10_000_000, seed=13)
    return wl.replace(**kw)


FIG12_MASSES = (5.0, 10.0, 20.0, 40.0)      # mg/cm^2


def fig12(m0_mg: float, **kw) -> Workload:
    """A Monte Carlo case of the comparison with the single-scattering model
    (Section III.B, Fig. 12): beta = 10, log-normal d_m = 1.5 um, sigma = 0.5,
    area mass m0_mg (mg/cm^2); Mie 3+9i at 1550 nm, every upward photon
    counted, 1200 bins over 0-8000 m/s at 1 us, 1e7 packets."""
    wl = Workload(
        name="fig12-m0-%g" % m0_mg, m0=m0_mg * MG_CM2, beta=10.0, v_max=0.0, d_m=1.5 * UM,
        sigma_ln=0.5, phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=256),
        r_ap=0.0, cone_alpha=math.pi / 2, t_snap=(1.0 * US,), n_bins=1200, v_lo=0.0,
        v_hi=8000.0, n_packets=10_000_000, seed=12)
    return wl.replace(**kw)


def fig4(**kw) -> Workload:
    """The convergence and timing case of Section II.D (Fig. 4; the paper's
    CPU / GPU timings are quoted on it): tin, beta = 10, log-normal d_m = 1.5
    um, sigma = 0.5, m0 = 20 mg/cm^2, lambda = 1550 nm, Mie phase function;
    every upward photon is counted; 1e7 photons, the paper's 1000 layers;
    600 bins over 0-8000 m/s at 1 us."""
    wl = Workload(
        name="fig4", m0=20.0 * MG_CM2, beta=10.0, v_max=0.0, d_m=1.5 * UM, sigma_ln=0.5,
        phase=Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=256),
        r_ap=0.0, cone_alpha=math.pi / 2, t_snap=(1.0 * US,), n_bins=600, v_lo=0.0,
        v_hi=8000.0, n_packets=10_000_000, seed=9, n_layers=1000)
    return wl.replace(**kw)
