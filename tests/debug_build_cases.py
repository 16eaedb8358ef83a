"""Cases for the debug build (libpdv_debug.so), run by tests/test_gpu_debug.py
in a child process with PDV_LIBRARY=debug (a process loads one of the two
libraries). The file name keeps pytest from collecting it in the main run.

* Every path (FP32 and FP64 transport, batch graph, serving, fixed scratch,
  layer stepping) on the parity workloads records no failed index check, and
  still meets the parity bar against the FP64 oracle.
* PDV_TEST_DEBUG_CHECK evaluates one check one past the end of the tally
  (without the access): the call returns PDV_EDEBUG with that record, the
  context stays usable, and pdv_debug_get(reset) clears the record.
* The path trace of the first packets has the oracle's vertices: the same
  kinds in the same order on packets with equal event counts, and the same
  positions, velocities and directions within the arithmetic's rounding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

from parity_helpers import compare

pytestmark = pytest.mark.gpu

WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


@pytest.fixture(scope="module")
def ctx():
    assert pdv.library_path().endswith("libpdv_debug.so")
    c = pdv.Context(0)
    yield c
    c.close()


def clean(ctx):
    d = pdv.pdv_debug_get(ctx.handle)
    assert d["debug_build"] == 1
    assert d["violations"] == 0, d


def test_debug_library_loaded(ctx):
    clean(ctx)


VARIANTS = {
    "cfg1": dict(),
    "tabulated": dict(profile_kind="tabulated", prof_v=[2100.0, 2600.0, 3000.0, 4200.0],
                      prof_f=[3.0, 1.0, 2.0, 0.2], v_max=0.0, m0=1 * W.MG_CM2),
    "specular": dict(surface_mode=2, reflectivity=0.3),
    "maxev2": dict(max_events=2),
    "onebin": dict(n_bins=1, v_lo=1000.0, v_hi=5000.0),
    "open_aperture_cone_4t": dict(r_ap=0.0, cone_alpha=0.5, t_snap=(1.0e-6, 0.7e-6, 2.0e-6, 4.0e-6)),
    "detect_all_3t": dict(r_ap=0.0, cone_alpha=2.0, t_snap=(0.5e-6, 1.0e-6, 3.0e-6)),
    "horizontal": dict(horizontal_launch=True, r_ap=0.0, cone_alpha=2.0),
    "implicit": dict(implicit_capture=True),
}


@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_parity_under_index_checks(ctx, precision, name):
    wl = W.cfg1(n_packets=20000, **WIDE).replace(**VARIANTS[name])
    ref = O.simulate(wl, packets=True)
    cloud = pdv.Cloud(ctx, wl)
    out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True)
    cloud.close()
    clean(ctx)
    compare(out, ref, wl, precision)


def test_mie_cloud_and_layer_stepping_under_index_checks(ctx):
    """A Mie table (non-uniform work in the phase search) at 7 times, and
    the paper's layer stepping."""
    wl = W.cfg2(n_packets=20000, t_snap=tuple(np.linspace(0.5, 5.0, 7) * W.US), **WIDE)
    table = O.phase_table(wl)
    ref = O.simulate(wl, packets=True, table=table)
    cloud = pdv.Cloud(ctx, wl, table=table)
    out = pdv.simulate_spectrum(ctx, cloud, wl, packets=True)
    clean(ctx)
    compare(out, ref, wl, "fp32")
    ws = wl.replace(n_packets=4000, n_layers=200)
    ref_s = O.simulate(ws, packets=True, table=table)
    out_s = pdv.simulate_spectrum(ctx, cloud, ws, packets=True)
    cloud.close()
    clean(ctx)
    assert np.mean(out_s["packets"]["n_events"] == ref_s["packets"]["n_events"]) >= 0.999


@pytest.mark.parametrize("hist_mode", [1, 2])
def test_batch_serving_and_fixed_scratch_under_index_checks(ctx, hist_mode):
    import torch
    wls = [W.cfg1(n_packets=30000 + 5000 * i, seed=11 + i, **WIDE) for i in range(3)]
    wls[2] = wls[2].replace(r_ap=0.0, cone_alpha=2.0, t_snap=(1e-6, 2e-6))
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    ctx.set_tuning(hist_mode=hist_mode)
    try:
        batch = pdv.simulate_batch(ctx, clouds, wls)
        clean(ctx)
        alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
        for a, b in zip(batch, alone):
            assert np.array_equal(a["raw"], b["raw"])
        reqs = [pdv.Request(c, w) for c, w in zip(clouds, wls)]
        tickets = [pdv.pdv_submit(ctx.handle, r.c) for r in reqs]
        for t in tickets:
            while pdv.pdv_poll(ctx.handle, t, 100000) != pdv.PDV_OK:
                pass
        clean(ctx)
        for r, b in zip(reqs, alone):
            assert np.array_equal(r.raw, b["raw"])
        wl = wls[0]
        dev = {"spectrum": torch.zeros(len(wl.t_snap) * wl.n_bins, dtype=torch.float64, device="cuda"),
               "raw": torch.zeros(len(wl.t_snap) * (wl.n_bins + 2), dtype=torch.int64, device="cuda")}
        req = pdv.Request(clouds[0], wl, device_out=dev)
        torch.cuda.synchronize()
        pdv.pdv_simulate_spectrum_static(ctx.handle, req.c)
        clean(ctx)
        got = dev["raw"].cpu().numpy().view(np.uint64).reshape(alone[0]["raw"].shape)
        assert np.array_equal(got, alone[0]["raw"])
    finally:
        ctx.set_tuning()
        for c in clouds:
            c.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("detect_all", [False, True])
def test_check_failure_is_reported_and_cleared(ctx, precision, detect_all):
    kw = dict(r_ap=0.0, cone_alpha=2.0) if detect_all else dict(WIDE, t_snap=(1e-6, 2e-6))
    wl = W.cfg1(n_packets=5000, **kw)
    cloud = pdv.Cloud(ctx, wl)
    with pytest.raises(pdv.PdvError) as e:
        pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, debug_check=True)
    assert e.value.status == pdv.PDV_EDEBUG
    d = pdv.pdv_debug_get(ctx.handle, reset=True)
    # one row when every time detects alike (FP32), else one row per time
    rows = 1 if (detect_all and precision == "fp32") else len(wl.t_snap)
    n = rows * (wl.n_bins + 3)
    assert d["violations"] == 1 and d["site_name"] == "selftest", d
    assert d["index"] == n and d["bound"] == n, d
    clean(ctx)
    out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision)    # still usable
    clean(ctx)
    assert out["counters"][0][0] == wl.n_packets
    cloud.close()


TRACE_CASES = {
    "cfg1": dict(),
    "specular": dict(surface_mode=2, reflectivity=0.3),
    "lambert": dict(surface_mode=1, reflectivity=1.0),
    "albedo0": dict(phase=W.Phase(albedo=0.0)),
    "maxev2": dict(max_events=2),
    "horizontal": dict(horizontal_launch=True, r_ap=0.0, cone_alpha=2.0),
    "implicit": dict(implicit_capture=True),
    "tabulated": dict(profile_kind="tabulated", prof_v=[2100.0, 2600.0, 3000.0, 4200.0],
                      prof_f=[3.0, 1.0, 2.0, 0.2], v_max=0.0, m0=1 * W.MG_CM2),
}
# FP64: the same arithmetic in another order, its rounding grown over the
# walk, and for a tabulated profile the linear interpolation of the 2048-node
# velocity table (a few 1e-7 of v_fs) where the oracle inverts the profile
# itself; directions do not see the table. FP32: binary32 rounding of the
# walk (direction, lateral sum,
# fixed-point depth) grown over a few events; a packet whose apparent velocity
# is sensitive to rounding (the oracle's FP64 re-runs with binary32-sized
# errors spread it beyond 1e-5 v_fs) is held to its kinds only, as its later
# vertices move with that sensitivity.
TRACE_TOL = {"fp64": (1e-6, 1e-7), "fp32": (2e-4, 2e-4)}


@pytest.mark.parametrize("name", list(TRACE_CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_path_trace_matches_oracle(ctx, precision, name):
    n_tr, max_v = 200, 48
    wl = W.cfg1(n_packets=2000, **WIDE).replace(**TRACE_CASES[name])
    ref = O.simulate(wl, packets=True, n_trace=n_tr, max_vertices=max_v)
    cloud = pdv.Cloud(ctx, wl)
    out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True,
                                trace=(n_tr, max_v))
    cloud.close()
    clean(ctx)
    g, o = out["trace"], ref["trace"]
    pg, po = out["packets"][:n_tr], ref["packets"][:n_tr]
    same = pg["n_events"] == po["n_events"]
    assert same.mean() >= 0.99
    assert np.array_equal(g["kind"][same], o["kind"][same])
    # a path: the launch, one vertex per event, and the escape if it escaped
    n_vtx = (g["kind"] >= 0).sum(axis=1)
    want = np.minimum(1 + pg["n_events"].astype(np.int64) + (pg["fate"] == 1), max_v)
    assert np.array_equal(n_vtx, want), "vertex count"
    assert np.all(g["kind"][:, 0] == 0) and np.all(g["event"][g["kind"] > 0] > 0)
    stable = same if precision == "fp64" else same & (po["v_app_spread"] <= 1e-5 * wl.v_fs)
    assert stable.sum() >= 0.8 * n_tr, int(stable.sum())
    used = (g["kind"] >= 0) & stable[:, None]
    rel, abs_u = TRACE_TOL[precision]
    v_err = np.abs(g["v"] - o["v"])[used]
    assert v_err.max() <= rel * wl.v_fs, v_err.max()
    # positions against the probe distance; the escape vertex's position moves
    # with its direction over the vacuum flight, by 1 / |u_z|
    lever = np.where(g["kind"] == 3, 1.0 / np.maximum(np.abs(o["uz"]), 1e-3), 1.0)
    for f in ("x", "y", "z"):
        err = (np.abs(g[f] - o[f]) / lever)[used]
        assert err.max() <= rel * wl.z_probe, (f, err.max())
    # directions after each vertex but the last of each path (the final
    # vertex of an absorbed packet keeps whatever direction the walk held)
    last = np.zeros_like(used)
    last[np.arange(n_tr), np.maximum(n_vtx - 1, 0)] = True
    mid = used & ~last
    for f in ("ux", "uy", "uz"):
        err = np.abs(g[f] - o[f])[mid]
        assert err.max() <= abs_u, (f, err.max())


def test_trace_arguments(ctx):
    with pytest.raises(pdv.PdvError):
        pdv.pdv_debug_set_trace(ctx.handle, 70000, 8, np.zeros((1, 1), pdv.TRACE_DTYPE))
    with pytest.raises(pdv.PdvError):
        pdv.pdv_debug_set_trace(ctx.handle, 4, 0, np.zeros((4, 1), pdv.TRACE_DTYPE))
    # more traced packets than the request has: the extra rows stay empty
    wl = W.cfg1(n_packets=10, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    out = pdv.simulate_spectrum(ctx, cloud, wl, packets=True, trace=(16, 8))
    cloud.close()
    assert np.all(out["trace"]["kind"][10:] == -1)
    assert np.all(out["trace"]["kind"][:10, 0] == 0)
    clean(ctx)
