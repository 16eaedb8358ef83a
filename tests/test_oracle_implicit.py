"""Pins for the oracle's implicit capture with Russian roulette (a weight
variant of Section II.B step (4); the paper's own walk takes the analog choice
of Eq. 11). What fixes it without re-reading its code:
  - omega = 1 with a perfect mirror keeps every weight at 2^32: the walk is
    the analog walk, bit for bit;
  - omega = 0 absorbs the whole weight at the first interaction, which is
    what the analog walk absorbs;
  - an escape after k particle scatters carries k kept fractions of the
    weight, about 2^32 omega^k 16^j with j its roulette survivals, when the
    surface reflects fully, and one roulette in 16 is survived;
  - the weight ledger closes exactly, roulette included;
  - the tallies' expectations equal the analog walk's."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import workloads as W

TWO32 = 2**32
RR_W = 1 << 22          # roulette threshold (2^-10 of the launch weight)
RR_M = 16               # survival one in 16, at 16 times the weight


def _c(res, s=0):
    return O.counters_dict(res["counters"][s])


def _ledger_closes(c):
    out = (c["w_detected"] + c["w_under"] + c["w_over"] + c["w_escaped_undetected"] +
           c["w_absorbed_particle"] + c["w_absorbed_surface"] + c["w_truncated"] +
           c["w_roulette_dropped"])
    return out == c["launched"] * TWO32 + c["w_roulette_gained"]


def _pair(wl):
    a = O.simulate(wl, n_threads=4, packets=True)
    b = O.simulate(wl.replace(implicit_capture=True), n_threads=4, packets=True)
    return a, b


def test_omega_one_and_full_mirror_is_the_analog_walk():
    wl = W.cfg1(n_packets=20000, phase=W.Phase(albedo=1.0), reflectivity=1.0,
                m0=3 * W.MG_CM2, r_ap=0.0, cone_alpha=2.0)
    a, b = _pair(wl)
    assert np.array_equal(a["packets"], b["packets"])
    assert np.array_equal(a["hist"], b["hist"])
    assert np.array_equal(a["counters"], b["counters"])
    assert _c(b)["w_roulette_dropped"] == 0 and _c(b)["w_roulette_gained"] == 0


def test_omega_zero_absorbs_the_analog_weight():
    wl = W.cfg1(n_packets=20000, phase=W.Phase(albedo=0.0), m0=2 * W.MG_CM2)
    a, b = _pair(wl)
    pa, pb = a["packets"], b["packets"]
    for f in ("n_events", "n_scatters", "n_surface", "v_app", "detect_mask"):
        assert np.array_equal(pa[f], pb[f]), f
    absorbed = pa["fate"] == O.FATE_ABS_PARTICLE
    assert absorbed.any()
    assert np.all(pb["fate"][absorbed] == O.FATE_DROPPED)
    assert np.all(pb["weight"][absorbed] == 0)
    assert np.array_equal(pa["fate"][~absorbed], pb["fate"][~absorbed])
    assert np.array_equal(a["hist"], b["hist"])
    assert np.array_equal(a["counters"], b["counters"])


def _walk_weight(k, omega_q):
    """Weight after k interactions of a packet that survived every roulette:
    keep the fraction omega_q / 2^24 of the weight, rounded to nearest, and
    multiply a weight that fell below the threshold by 16. Returns the weight
    and the number of roulettes survived."""
    w, n = TWO32, 0
    for _ in range(k):
        w = (w * omega_q + (1 << 23)) >> 24
        if w < RR_W:
            w *= RR_M
            n += 1
    return w, n


@pytest.mark.parametrize("albedo", [0.6, 0.93])
def test_weight_law_of_escapes_and_drops(albedo):
    """With a perfect mirror an escape after k scatters carries exactly the
    weight of k kept fractions (about 2^32 omega^k 16^j, j its survivals); a
    drop carries the kept fraction of the next interaction, below the
    threshold. One roulette in 16 is survived."""
    wl = W.cfg1(n_packets=20000, phase=W.Phase(albedo=albedo), reflectivity=1.0,
                m0=4 * W.MG_CM2, implicit_capture=True)
    r = O.simulate(wl, n_threads=4, packets=True)
    pk = r["packets"]
    oq = math.floor(albedo * 2**24 + 0.5)
    esc = pk["fate"] == O.FATE_ESCAPED
    drop = pk["fate"] == O.FATE_DROPPED
    assert esc.sum() > 1000 and drop.sum() > 1000
    assert esc.sum() + drop.sum() == wl.n_packets
    survived = 0
    for p in pk[esc]:
        k = int(p["n_scatters"])
        w, n = _walk_weight(k, oq)
        assert int(p["weight"]) == w, (k, int(p["weight"]), w)
        assert abs(math.log(w / (TWO32 * (oq / 2**24) ** k), RR_M) - n) < 1e-3
        survived += n
    for p in pk[drop]:
        w, n = _walk_weight(int(p["n_scatters"]), oq)
        wn = (w * oq + (1 << 23)) >> 24
        assert int(p["weight"]) == wn < RR_W
        survived += n
    n_rr = survived + int(drop.sum())
    assert abs(survived / n_rr - 1 / RR_M) < 4 * math.sqrt((1 / RR_M) * (1 - 1 / RR_M) / n_rr)
    c = _c(r)
    assert c["w_roulette_dropped"] == int(pk["weight"][drop].sum())
    assert c["w_roulette_gained"] > 0


@pytest.mark.parametrize("kw", [
    dict(),
    dict(surface_mode=1, reflectivity=0.8, m0=4 * W.MG_CM2),
    dict(surface_mode=2, reflectivity=0.37, cone_alpha=2.0, r_ap=0.0),
    dict(phase=W.Phase(albedo=0.97), m0=6 * W.MG_CM2, max_events=40),
    dict(t_snap=(0.5 * W.US, 1.0 * W.US, 4.0 * W.US), v_lo=2500.0, v_hi=3500.0),
])
def test_ledger_and_event_bookkeeping(kw):
    wl = W.cfg1(n_packets=20000, implicit_capture=True, **kw)
    r = O.simulate(wl, n_threads=4, packets=True)
    pk = r["packets"]
    for s in range(len(wl.t_snap)):
        c = _c(r, s)
        assert _ledger_closes(c), c
        assert c["launched"] == wl.n_packets
    c = _c(r)
    n_drop = int(np.sum(pk["fate"] == O.FATE_DROPPED))
    assert c["events"] == c["scatters"] + c["surface_hits"] + n_drop
    assert c["events"] == int(pk["n_events"].sum())
    assert c["escapes"] == int(np.sum(pk["fate"] == O.FATE_ESCAPED))
    assert c["truncated"] == int(np.sum(pk["fate"] == O.FATE_TRUNCATED))
    if wl.max_events == 40:
        assert c["truncated"] > 0


def _z(x, y):
    d = x.mean() - y.mean()
    return abs(d) / math.sqrt(x.var() / len(x) + y.var() / len(y) + 1e-300)


@pytest.mark.parametrize("albedo,m0", [(0.6, 2.0), (0.9, 5.0)])
def test_expectations_equal_the_analog_walk(albedo, m0):
    """Independent streams (different seeds): the means of the escaped weight,
    the detected weight and the detected weight's first velocity moment agree
    within 5 standard errors."""
    wl = W.cfg1(n_packets=60000, phase=W.Phase(albedo=albedo), m0=m0 * W.MG_CM2,
                r_ap=0.0, cone_alpha=2.0)
    a = O.simulate(wl, n_threads=4, packets=True)["packets"]
    b = O.simulate(wl.replace(implicit_capture=True, seed=wl.seed + 101), n_threads=4,
                   packets=True)["packets"]

    def tallies(p):
        w = p["weight"].astype(np.float64) / TWO32
        esc = np.where(p["fate"] == O.FATE_ESCAPED, w, 0.0)
        det = np.where(p["detect_mask"] & 1, w, 0.0)
        return esc, det, det * p["v_app"] / wl.v_fs

    for x, y in zip(tallies(a), tallies(b)):
        assert _z(x, y) < 5.0, (x.mean(), y.mean(), _z(x, y))
    # implicit capture lowers the variance of the escaped weight
    assert tallies(b)[0].var() < tallies(a)[0].var()


def test_layer_stepping_rejects_implicit_capture():
    wl = W.cfg1(n_packets=100, n_layers=100, implicit_capture=True)
    with pytest.raises(ValueError):
        O.simulate(wl, n_threads=1)
