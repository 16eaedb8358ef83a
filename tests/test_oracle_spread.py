"""Pins of the oracle's rounding-sensitivity estimate (``v_app_spread``): the
largest change of a packet's v_app over FP64 re-runs with random errors of the
size of binary32 roundings injected into every flight and every new direction.
The GPU parity bar allows the FP32 path four times this spread on top of 1e-5,
so these tests fix what the spread is before any GPU result is seen."""
import numpy as np

from oracle import oracle as O
from paper_2012_00963_gb300 import workloads as W

WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


def _run(wl, **kw):
    return O.simulate(wl, packets=True, table=O.phase_table(wl), **kw)["packets"]


def test_zero_perturbation_gives_zero_spread():
    wl = W.cfg2(n_packets=3000, t_snap=(1e-6,), **WIDE)
    p = _run(wl, spread_sd=(0.0, 0.0, 0.0))
    assert np.all(p["v_app_spread"] == 0.0)
    assert np.all(p["n_unstable"] == 0)


def test_re_runs_leave_the_walk_unchanged():
    wl = W.cfg3(n_packets=4000, r_ap=0.0, cone_alpha=2.0)
    tb = O.phase_table(wl)
    a = O.simulate(wl, packets=True, table=tb, spread_runs=0)
    b = O.simulate(wl, packets=True, table=tb, spread_runs=3)
    for k in ("n_events", "n_scatters", "fate", "weight", "v_app", "detect_mask"):
        assert np.array_equal(a["packets"][k], b["packets"][k]), k
    assert np.array_equal(a["hist"], b["hist"]) and np.array_equal(a["counters"], b["counters"])
    assert np.all(a["packets"]["v_app_spread"] == 0.0)


def test_spread_is_linear_in_the_perturbation_size():
    """First-order sensitivity: doubling every error doubles the spread of a
    well-conditioned packet (the same random draws, scaled)."""
    wl = W.cfg2(n_packets=4000, t_snap=(1e-6,), **WIDE)
    a = _run(wl)
    b = _run(wl, spread_sd=tuple(2.0 * x for x in O.SPREAD_SD))
    m = (a["v_app_spread"] > 0) & (a["n_unstable"] == 0) & (b["n_unstable"] == 0)
    assert m.sum() > 1000
    r = b["v_app_spread"][m] / a["v_app_spread"][m]
    assert 1.9 < np.median(r) < 2.1, np.median(r)


def test_exact_specular_echo_spread_is_one_rounding():
    """Empty cloud, specular surface: every packet returns with v_app = v_fs
    = (u_z,out - u_z,in) v_fs / 2 after one turn, so its spread is the stored
    u_z's error times v_fs / 2, with nothing to amplify it."""
    wl = W.cfg1(n_packets=2000, m0=0.0, surface_mode=2, v_lo=1900.0, v_hi=2100.0, n_bins=10)
    p = _run(wl)
    assert np.all(p["v_app"] == wl.v_fs)
    s = p["v_app_spread"] / wl.v_fs
    sd = (O.SPREAD_SD[1] + O.SPREAD_SD[2]) * 2.0**-24
    assert np.all(s <= 3.0 * sd) and np.median(s) > 0.05 * sd, (np.median(s), s.max())


def test_single_backscatter_spread_is_rounding_sized():
    """A thin sheet at a single velocity (tau << 1): a detected packet turns
    once, v_app = (1 + u_z,out) v0 / 2, and its spread is of the order of the
    injected direction error times v0."""
    v0 = 3000.0
    wl = W.cfg1(n_packets=20000, m0=0.05 * W.MG_CM2, profile_kind="tabulated",
                prof_v=[v0 - 0.5, v0 + 0.5], prof_f=[1.0, 1.0], v_max=0.0, reflectivity=0.0,
                phase=W.Phase(albedo=1.0), r_ap=0.0, cone_alpha=2.0, v_lo=0.0, v_hi=4000.0)
    p = _run(wl)
    one = (p["n_scatters"] == 1) & (p["n_surface"] == 0) & (p["fate"] == O.FATE_ESCAPED)
    assert one.sum() > 20
    u = 2.0**-24
    s = p["v_app_spread"][one] / v0
    sd = O.SPREAD_SD[1] + O.SPREAD_SD[2]
    assert np.all(s <= 5.0 * sd * u) and np.median(s) > 0.05 * sd * u, (s.min(), np.median(s), s.max())


def test_spread_does_not_depend_on_threads():
    wl = W.cfg2(n_packets=3000, t_snap=(1e-6, 2e-6), **WIDE)
    tb = O.phase_table(wl)
    a = O.simulate(wl, packets=True, table=tb, n_threads=1)["packets"]
    b = O.simulate(wl, packets=True, table=tb, n_threads=5)["packets"]
    assert np.array_equal(a["v_app_spread"], b["v_app_spread"])
    assert np.array_equal(a["n_unstable"], b["n_unstable"])


def test_layer_stepping_has_a_spread():
    wl = W.cfg1(n_packets=2000, n_layers=200, **WIDE)
    p = _run(wl)
    moved = p["n_scatters"] > 0
    assert np.all(p["v_app_spread"][moved & (p["n_unstable"] == 0)] > 0.0)
