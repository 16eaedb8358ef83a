"""Implicit capture with Russian roulette (PDV_IMPLICIT_CAPTURE) through the C
ABI against the FP64 oracle's same variant: packet walks, integer weights,
spectra and the roulette's weight ledger, in both precisions; the reduction to
the analog walk at omega = 1 with a perfect mirror; batches that mix the two
schemes; and the rejection of the flag with layer stepping."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

from parity_helpers import compare as _compare, conserved

pytestmark = pytest.mark.gpu

WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


def compare(out, ref, wl, precision):
    """The packet-level bar of parity_helpers.compare. Long walks need no bar of
    their own: the oracle's perturbed re-runs follow every scattering of the
    walk, so each packet's rounding sensitivity grows with its walk."""
    return _compare(out, ref, wl, precision)


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def run_pair(ctx, wl, precision, table=None):
    ref = O.simulate(wl, packets=True, table=table)
    cloud = pdv.Cloud(ctx, wl, table=table)
    try:
        out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True)
    finally:
        cloud.close()
    return out, ref


def check_weights(out, ref, precision):
    """Weights are integers decided by the walk: every packet whose walk ended
    alike (events, scatters, surface hits, fate) carries the same weight."""
    a, b = out["packets"], ref["packets"]
    walk = ((a["n_events"] == b["n_events"]) & (a["n_scatters"] == b["n_scatters"]) &
            (a["n_surface"] == b["n_surface"]) & (a["fate"] == b["fate"]))
    assert walk.mean() >= (0.999 if precision == "fp64" else 0.998), walk.mean()
    assert np.mean(a["weight"][walk] == b["weight"][walk]) >= 0.9995
    ca, cb = pdv.counters_dict(out["counters"][0]), O.counters_dict(ref["counters"][0])
    for k in ("w_roulette_dropped", "w_roulette_gained", "w_absorbed_particle"):
        assert abs(ca[k] - cb[k]) <= 2e-3 * max(cb[k], 1) + 2**33, (k, ca[k], cb[k])
    assert ca["w_roulette_dropped"] == int(a["weight"][a["fate"] == 5].sum())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg1_hg_cloud(ctx, precision):
    wl = W.cfg1(n_packets=200000, m0=3 * W.MG_CM2, implicit_capture=True, **WIDE)
    out, ref = run_pair(ctx, wl, precision)
    compare(out, ref, wl, precision)
    check_weights(out, ref, precision)
    assert pdv.counters_dict(out["counters"][0])["w_roulette_gained"] > 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg2_lognormal_mie_multi_snapshot(ctx, precision):
    wl = W.cfg2(n_packets=40000, t_snap=tuple(np.linspace(0.5, 5.0, 7) * W.US),
                implicit_capture=True, **WIDE)
    out, ref = run_pair(ctx, wl, precision, table=O.phase_table(wl))
    compare(out, ref, wl, precision)
    check_weights(out, ref, precision)


@pytest.mark.parametrize("kw", [
    dict(phase=W.Phase(albedo=0.93), m0=6 * W.MG_CM2, r_ap=0.0, cone_alpha=2.0),
    dict(surface_mode=1, reflectivity=0.8, m0=4 * W.MG_CM2),
    dict(surface_mode=2, reflectivity=0.37),
    dict(phase=W.Phase(albedo=0.0)),
    dict(phase=W.Phase(albedo=0.97), m0=6 * W.MG_CM2, max_events=40),
], ids=["albedo093_open", "lambert", "specular", "albedo0", "maxev40"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_variants(ctx, precision, kw):
    wl = W.cfg1(n_packets=50000, implicit_capture=True, **WIDE).replace(**kw)
    out, ref = run_pair(ctx, wl, precision)
    compare(out, ref, wl, precision)
    check_weights(out, ref, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_omega_one_and_full_mirror_is_the_analog_walk(ctx, precision):
    wl = W.cfg1(n_packets=100000, phase=W.Phase(albedo=1.0), reflectivity=1.0,
                m0=3 * W.MG_CM2, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    try:
        a = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True)
        b = pdv.simulate_spectrum(ctx, cloud, wl.replace(implicit_capture=True),
                                  precision=precision, packets=True)
    finally:
        cloud.close()
    assert np.array_equal(a["raw"], b["raw"])
    assert np.array_equal(a["counters"], b["counters"])
    assert np.array_equal(a["packets"], b["packets"])


def test_batch_mixes_analog_and_implicit_sets(ctx):
    sets = W.cfg4_sets(n_sets=4, seed=45, n_min=2e4, n_max=2e5)
    wls = [s.replace(phase=W.Phase(kind="hg", g=0.6 + 0.02 * i, albedo=0.55 + 0.1 * i),
                     r_ap=2e-3, cone_alpha=0.4, implicit_capture=bool(i % 2))
           for i, s in enumerate(sets)]
    wls[3] = wls[3].replace(precision="fp64")
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    try:
        alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
        batch = pdv.simulate_batch(ctx, clouds, wls)
    finally:
        for c in clouds:
            c.close()
    for w, a, b in zip(wls, alone, batch):
        assert np.array_equal(a["raw"], b["raw"])
        assert np.array_equal(a["counters"], b["counters"])
        assert conserved(a["counters"][0])
        if not w.implicit_capture:
            assert pdv.counters_dict(a["counters"][0])["w_roulette_gained"] == 0


def test_layer_stepping_rejects_the_flag(ctx):
    wl = W.cfg1(n_packets=1000, n_layers=100, implicit_capture=True)
    cloud = pdv.Cloud(ctx, wl)
    try:
        with pytest.raises(pdv.PdvError):
            pdv.simulate_spectrum(ctx, cloud, wl)
    finally:
        cloud.close()


def test_packet_ranges_add_up_exactly(ctx):
    """Checkpoint/resume with implicit capture: tallies and every counter of
    [0, k) and [k, N) sum to those of [0, N)."""
    wl = W.cfg1(n_packets=200000, m0=3 * W.MG_CM2, implicit_capture=True, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    try:
        full = pdv.simulate_spectrum(ctx, cloud, wl)
        a = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=77777)
        b = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=200000 - 77777, packet_begin=77777)
    finally:
        cloud.close()
    assert np.array_equal(full["raw"], a["raw"] + b["raw"])
    for k, name in enumerate(pdv.COUNTER_NAMES):   # every counter is a sum over packets
        assert full["counters"][0][k] == a["counters"][0][k] + b["counters"][0][k], name


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_packet_and_ragged_tail(ctx, precision):
    for n, begin in ((1, 0), (1, 4321), (5003, 999)):
        wl = W.cfg1(n_packets=n, m0=3 * W.MG_CM2, implicit_capture=True, **WIDE)
        ref = O.simulate(wl, packets=True, packet_begin=begin)
        cloud = pdv.Cloud(ctx, wl)
        try:
            out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True,
                                        packet_begin=begin)
        finally:
            cloud.close()
        same = out["packets"]["n_events"] == ref["packets"]["n_events"]
        assert same.mean() >= (1.0 if n == 1 else 0.999)
        assert np.array_equal(out["packets"]["weight"][same], ref["packets"]["weight"][same])
        assert conserved(out["counters"][0])
