"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs: packet-level event counts and apparent velocities, per-bin spectra,
detected weight, exact weight conservation; both the FP32 persistent path and
the plain FP64 path, on the paper's workload shapes and on edge cases."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

from parity_helpers import compare, conserved, v_app_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def run_pair(ctx, wl, precision, table=None, **kw):
    ref = O.simulate(wl, packets=True, table=table)
    cloud = pdv.Cloud(ctx, wl, table=table)
    try:
        out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True, **kw)
    finally:
        cloud.close()
    return out, ref


# ------------------------------------------------------------------ tables
@pytest.mark.parametrize("m,d,sig,n_size", [(3 + 9j, 3.0, 0.5, 256), (3 + 9j, 1.0, 0.0, 1),
                                            (1.55 + 0.0j, 1.2, 0.0, 1), (1.5 + 0.1j, 0.8, 0.3, 64)])
def test_mie_table_matches_oracle(ctx, m, d, sig, n_size):
    th, p, q, a, g = ctx.mie_table(m, 1550.0, d, sig, n_size, 1801)
    tho, po, qo, ao, go = O.mie_table(m, 1550e-9, d * 1e-6, sig, 1801, n_size)
    assert np.array_equal(th, tho) or np.allclose(th, tho, rtol=0, atol=1e-15)
    assert np.allclose(p, po, rtol=1e-11, atol=0)
    assert q == pytest.approx(qo, rel=1e-12)
    assert a == pytest.approx(ao, rel=1e-12)
    assert g == pytest.approx(go, rel=1e-11)


def test_cloud_constants_match_oracle(ctx):
    for wl in (W.cfg1(), W.cfg2(), W.cfg3()):
        cloud = pdv.Cloud(ctx, wl, table=O.phase_table(wl))
        info = cloud.info()
        c = O.Problem(wl).constants()
        cq, g_tab = O.phase_cdf(*O.phase_table(wl)[:2])
        cloud.close()
        assert info["tau_tot"] == pytest.approx(c["tau_tot"], rel=1e-14)
        assert info["v_top"] == pytest.approx(c["v_top"], rel=1e-15)
        assert info["g_table"] == pytest.approx(g_tab, rel=1e-12)


# ------------------------------------------------------------------ workloads
WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg1_hg_cloud(ctx, precision):
    wl = W.cfg1(n_packets=200000, **WIDE)
    out, ref = run_pair(ctx, wl, precision)
    compare(out, ref, wl, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg1_as_configured(ctx, precision):
    """The benchmark's first cloud with its own aperture (1 mm, 0.1 rad)."""
    wl = W.cfg1(n_packets=100000)
    out, ref = run_pair(ctx, wl, precision)
    compare(out, ref, wl, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg2_lognormal_mie_multi_snapshot(ctx, precision):
    """Log-normal Mie cloud at 7 snapshot times (one transport per packet,
    detection at every time) against per-snapshot oracle transports."""
    wl = W.cfg2(n_packets=40000, t_snap=tuple(np.linspace(0.5, 5.0, 7) * W.US), **WIDE)
    out, ref = run_pair(ctx, wl, precision, table=O.phase_table(wl))
    compare(out, ref, wl, precision)
    assert np.array_equal(out["packets"]["detect_mask"] != 0, ref["packets"]["detect_mask"] != 0) \
        or np.mean(out["packets"]["detect_mask"] == ref["packets"]["detect_mask"]) > 0.999


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cfg3_heavy_multiple_scattering(ctx, precision):
    """20 mg/cm^2 of 1 um spheres (Mie optical depth ~109)."""
    wl = W.cfg3(n_packets=20000, r_ap=0.0, cone_alpha=2.0)
    out, ref = run_pair(ctx, wl, precision, table=O.phase_table(wl))
    rep = compare(out, ref, wl, precision)
    assert out["counters"][0][1] > 5 * wl.n_packets   # many events per packet


@pytest.mark.parametrize("kw", [
    dict(surface_mode=1, reflectivity=1.0),
    dict(surface_mode=2, reflectivity=0.3),
    dict(reflectivity=0.0),
    dict(phase=W.Phase(albedo=1.0), m0=2 * W.MG_CM2),
    dict(phase=W.Phase(albedo=0.0)),
    dict(profile_kind="tabulated", prof_v=[2100.0, 2600.0, 3000.0, 4200.0],
         prof_f=[3.0, 1.0, 2.0, 0.2], v_max=0.0, m0=1 * W.MG_CM2),
    dict(beta=10.0, v_max=0.0, v_fs=1500.0, m0=3 * W.MG_CM2, v_hi=4000.0),
    dict(max_events=2),
    dict(n_bins=1, v_lo=1000.0, v_hi=5000.0),
    dict(phase=W.Phase(kind="mie_iso", m=3.0 + 9.0j, n_angle=1801, n_size=64), d_m=1.5e-6,
         sigma_ln=0.5, m0=2 * W.MG_CM2, v_max=0.0),
    dict(r_ap=0.0, cone_alpha=2.0),
    dict(r_ap=0.0, cone_alpha=2.0, t_snap=(0.5e-6, 1.0e-6, 3.0e-6)),
    dict(r_ap=0.0, cone_alpha=0.5, t_snap=(1.0e-6, 0.7e-6, 2.0e-6, 4.0e-6)),
    dict(horizontal_launch=True, r_ap=0.0, cone_alpha=2.0),
    dict(horizontal_launch=True, profile_kind="tabulated", prof_v=[2500.0, 4500.0],
         prof_f=[1.0, 1.0], v_max=0.0, m0=2 * W.MG_CM2, t_snap=(1.0e-6, 1.5e-6)),
], ids=["lambert", "specular", "R0", "albedo1", "albedo0", "tabulated", "steep", "maxev2",
        "onebin", "isotropic", "detect_all", "detect_all_3t", "open_aperture_cone_4t",
        "horizontal_exp_detect_all", "horizontal_flat_aperture_2t"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_variants(ctx, precision, kw):
    wl = W.cfg1(n_packets=50000, **WIDE).replace(**kw)
    out, ref = run_pair(ctx, wl, precision)
    compare(out, ref, wl, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_empty_cloud_specular_echo_is_exact(ctx, precision):
    wl = W.cfg1(n_packets=10000, m0=0.0, surface_mode=2, v_lo=1900.0, v_hi=2100.0, n_bins=10)
    out, ref = run_pair(ctx, wl, precision)
    pk = out["packets"]
    assert np.all(pk["v_app"] == wl.v_fs)
    c = pdv.counters_dict(out["counters"][0])
    assert c["detected"] == wl.n_packets
    assert c["w_detected"] == wl.n_packets * int(math.floor(0.6 * 2**32 + 0.5))
    compare(out, ref, wl, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_packet_and_ragged_tail(ctx, precision):
    """One packet, and a packet count that is not a multiple of the warp chunk,
    starting at an odd packet index."""
    for n, begin in ((1, 0), (1, 12345), (6397, 777)):
        wl = W.cfg1(n_packets=n, **WIDE)
        ref = O.simulate(wl, packets=True, packet_begin=begin)
        cloud = pdv.Cloud(ctx, wl)
        out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True,
                                    packet_begin=begin)
        cloud.close()
        assert np.array_equal(out["packets"]["n_events"], ref["packets"]["n_events"])
        assert pdv.counters_dict(out["counters"][0])["launched"] == n


# ------------------------------------------------------------------ properties
def test_packet_ranges_add_up_exactly(ctx):
    """Checkpoint/resume: tallies of [0, k) and [k, N) sum to those of [0, N)."""
    wl = W.cfg1(n_packets=300000, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    full = pdv.simulate_spectrum(ctx, cloud, wl)
    a = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=123457)
    b = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=300000 - 123457, packet_begin=123457)
    cloud.close()
    assert np.array_equal(full["raw"], a["raw"] + b["raw"])
    for k in (1, 2, 3, 4, 6, 10, 11, 12, 13):   # event and weight counters
        assert full["counters"][0][k] == a["counters"][0][k] + b["counters"][0][k]


def test_runs_are_bit_identical(ctx):
    wl = W.cfg2(n_packets=200000, t_snap=(1e-6, 3e-6))
    cloud = pdv.Cloud(ctx, wl)
    r1 = pdv.simulate_spectrum(ctx, cloud, wl)
    r2 = pdv.simulate_spectrum(ctx, cloud, wl)
    cloud.close()
    assert np.array_equal(r1["raw"], r2["raw"])
    assert np.array_equal(r1["counters"], r2["counters"])


# Request variants for the build check below: whether the FP32 transport
# without packet records runs the build compiled for the common configuration
# (exponential law, node angle table, vertical launch, uniform-angle wall with
# R < 1), and the workload change.
BUILDS = {
    "cfg1": (True, lambda: W.cfg1(n_packets=100000, **WIDE)),
    "cfg2_mie_5t": (True, lambda: W.cfg2(n_packets=100000, t_snap=(0.5e-6, 1e-6, 2e-6, 3.5e-6, 5e-6),
                                         **WIDE)),
    "detect_all_3t": (True, lambda: W.cfg1(n_packets=100000, r_ap=0.0, cone_alpha=2.0,
                                           t_snap=(0.5e-6, 1e-6, 3e-6))),
    "implicit": (True, lambda: W.cfg1(n_packets=100000, implicit_capture=True, **WIDE)),
    "albedo0": (True, lambda: W.cfg1(n_packets=100000, phase=W.Phase(albedo=0.0), **WIDE)),
    "maxev3": (True, lambda: W.cfg1(n_packets=100000, max_events=3, **WIDE)),
    "R1": (False, lambda: W.cfg1(n_packets=100000, reflectivity=1.0, **WIDE)),
    "coarse_table": (False, lambda: W.cfg1(n_packets=100000, phase=W.Phase(
        kind="table", theta=np.linspace(0.0, np.pi, 181),
        p=0.51 / (1.49 - 1.4 * np.cos(np.linspace(0.0, np.pi, 181))) ** 1.5, albedo=0.8, q_ext=2.0),
        **WIDE)),
    "specular": (False, lambda: W.cfg1(n_packets=100000, surface_mode=2, reflectivity=0.3, **WIDE)),
    "lambert": (False, lambda: W.cfg1(n_packets=100000, surface_mode=1, reflectivity=0.6, **WIDE)),
    "horizontal": (False, lambda: W.cfg1(n_packets=100000, horizontal_launch=True, r_ap=0.0,
                                         cone_alpha=2.0)),
    "tabulated": (False, lambda: W.cfg1(n_packets=100000, profile_kind="tabulated",
                                        prof_v=[2100.0, 2600.0, 3000.0, 4200.0],
                                        prof_f=[3.0, 1.0, 2.0, 0.2], v_max=0.0,
                                        m0=1 * W.MG_CM2, **WIDE)),
}


@pytest.mark.parametrize("name", list(BUILDS))
def test_common_configuration_build_matches_generic_build(ctx, name):
    """A request with packet records runs the generic build of the FP32
    transport (every switch of the set tested at run time); the same request
    without them runs the build compiled for the common configuration where
    the set has it. Both walk the same packets with the same arithmetic, so
    tallies and counters agree bit for bit, and the library reports which
    build ran."""
    fast, make = BUILDS[name]
    wl = make()
    cloud = pdv.Cloud(ctx, wl)
    plain = pdv.simulate_spectrum(ctx, cloud, wl)
    st_plain = ctx.stats()
    dump = pdv.simulate_spectrum(ctx, cloud, wl, packets=True)
    st_dump = ctx.stats()
    cloud.close()
    assert st_plain["transport_fast"] == int(fast) and st_dump["transport_fast"] == 0
    assert np.array_equal(plain["raw"], dump["raw"])
    assert np.array_equal(plain["counters"], dump["counters"])
    assert np.array_equal(plain["spectrum"], dump["spectrum"])


def test_device_outputs_match_host_outputs(ctx):
    torch = pytest.importorskip("torch")
    wl = W.cfg1(n_packets=100000, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    host = pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)
    ns, nb = len(wl.t_snap), wl.n_bins
    dev = {"spectrum": torch.zeros(ns * nb, dtype=torch.float64, device="cuda"),
           "raw": torch.zeros(ns * (nb + 2), dtype=torch.int64, device="cuda")}
    req = pdv.Request(cloud, wl, per_dv=True, device_out=dev)
    torch.cuda.synchronize()      # order torch's zero-fills before the context's stream
    pdv.pdv_simulate_spectrum(ctx.handle, req.c)
    torch.cuda.synchronize()
    cloud.close()
    assert np.array_equal(dev["spectrum"].cpu().numpy().reshape(ns, nb), host["spectrum"])
    assert np.array_equal(dev["raw"].cpu().numpy().view(np.uint64).reshape(ns, nb + 2), host["raw"])
    # per m/s: the spectrum integrates to the in-range detected fraction
    dv = (wl.v_hi - wl.v_lo) / nb
    assert host["spectrum"].sum() * dv == pytest.approx(host["raw"][0, 1:-1].sum() / 2**32 /
                                                         wl.n_packets, rel=1e-12)


def test_fp32_and_fp64_spectra_agree(ctx):
    wl = W.cfg2(n_packets=2_000_000, t_snap=(1e-6, 2.5e-6, 4e-6), **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    a = pdv.simulate_spectrum(ctx, cloud, wl, precision="fp32")
    b = pdv.simulate_spectrum(ctx, cloud, wl, precision="fp64")
    cloud.close()
    ha, hb = a["raw"].astype(float) / 2**32, b["raw"].astype(float) / 2**32
    assert np.max(np.abs(ha - hb) / np.sqrt(ha + hb + 1)) < 4


def test_invalid_requests_are_rejected(ctx):
    wl = W.cfg1(n_packets=1000)
    cloud = pdv.Cloud(ctx, wl)
    bad = [dict(snapshots=(0.0,)), dict(snapshots=(30e-6,))]
    for kw in bad:
        with pytest.raises(pdv.PdvError) as e:
            pdv.simulate_spectrum(ctx, cloud, wl, **kw)
        assert e.value.status == pdv.PDV_EINVAL
    r = pdv.Request(cloud, wl)
    r.c.n_bins = 0
    with pytest.raises(pdv.PdvError):
        pdv.pdv_simulate_spectrum(ctx.handle, r.c)
    r = pdv.Request(cloud, wl)
    r.c.n_packets = 0
    with pytest.raises(pdv.PdvError):
        pdv.pdv_simulate_spectrum(ctx.handle, r.c)
    with pytest.raises(pdv.PdvError):
        pdv.pdv_set_phase_table(cloud.handle, [0.0, 1.0], [1.0, 1.0], 2.0, 0.5)   # not 0..pi
    with pytest.raises(pdv.PdvError):
        pdv.Cloud(ctx, wl.replace(rho=-1.0))
    with pytest.raises(pdv.PdvError):
        pdv.Cloud(ctx, wl.replace(v_max=1000.0))
    cloud.close()


# ------------------------------------------------------------------ full size
def test_full_size_cfg2_sampled_packets(ctx):
    """The benchmark workload at full size (1e8 packets, 50 snapshots, FP32
    persistent launch): exact conservation at every snapshot, every packet
    launched, and packets sampled inside the full launch (dump variant, whose
    tallies are identical) equal the oracle's packet by packet under the
    per-packet v_app bar of parity_helpers."""
    torch = pytest.importorskip("torch")
    wl = W.cfg2()
    cloud = pdv.Cloud(ctx, wl)
    ns, nb, n = len(wl.t_snap), wl.n_bins, wl.n_packets
    full = pdv.simulate_spectrum(ctx, cloud, wl)
    for row in full["counters"]:
        assert conserved(row)
        assert pdv.counters_dict(row)["launched"] == n
    pk = torch.zeros(n * pdv.PACKET_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    dev = {"spectrum": torch.zeros(ns * nb, dtype=torch.float64, device="cuda"),
           "raw": torch.zeros(ns * (nb + 2), dtype=torch.int64, device="cuda"), "packets": pk}
    req = pdv.Request(cloud, wl, device_out=dev)
    torch.cuda.synchronize()      # the zero-fills above run on torch's stream, not the context's
    pdv.pdv_simulate_spectrum(ctx.handle, req.c)
    torch.cuda.synchronize()
    got_raw = dev["raw"].cpu().numpy().view(np.uint64).reshape(ns, nb + 2)
    diff = np.abs(got_raw.astype(np.float64) - full["raw"].astype(np.float64)) / 2**32
    assert np.array_equal(got_raw, full["raw"]), (diff.max(), int((diff > 0).sum()))
    recs = pk.view(-1, pdv.PACKET_DTYPE.itemsize)
    starts = [0, 31_415_926, n - 20000]
    table = O.phase_table(wl)
    got = np.concatenate([np.frombuffer(recs[s0:s0 + 20000].cpu().numpy().tobytes(),
                                        pdv.PACKET_DTYPE) for s0 in starts])
    refs = [O.simulate(wl, n_packets=20000, packet_begin=s0, packets=True, table=table)
            for s0 in starts]
    ref = {"packets": np.concatenate([r["packets"] for r in refs]),
           "hist": sum(r["hist"] for r in refs), "counters": sum(r["counters"] for r in refs)}
    a, b = got, ref["packets"]
    same = a["n_events"] == b["n_events"]
    assert same.mean() >= 0.999
    ok, checked, rep = v_app_check(a, b, wl.v_fs, "fp32")
    assert len(a) - rep["n_checked"] <= 0.001 * len(a), rep
    assert ok[checked].all(), rep
    assert np.mean(a["detect_mask"] == b["detect_mask"]) >= 0.999
    cloud.close()
    del pk, dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("seed,stream", [(11, 0), (2**63 + 12345, 7), (0xFFFFFFFF00000001, 2**31 + 3)],
                         ids=["small", "high_word", "both_words"])
def test_seed_and_stream_words(ctx, seed, stream):
    """Philox key = (seed_lo, seed_hi) and counter word 3 = stream id: seeds that
    use the high key word and large stream ids give the oracle's packets too,
    in the exact scheme and in the layer-stepping scheme."""
    for extra in (dict(), dict(n_layers=300)):
        wl = W.cfg1(n_packets=20000, seed=seed, stream_id=stream, **WIDE).replace(**extra)
        out, ref = run_pair(ctx, wl, "fp32")
        compare(out, ref, wl, "fp32")
