"""GPU parity of the paper's layer-stepping scheme (request field n_layers > 0:
steps of H / n_layers, Bernoulli pass per layer, interaction at the step's
end, acceptance-rejection angles) against the oracle's implementation of the
same scheme, packet by packet, through the C ABI. The bar is the one of the
exact scheme (``parity_helpers.compare``, FP32 criteria): the GPU keeps the
photon height as 62-bit fixed point, so its layer optical depths match the
oracle's FP64 ones to about 1e-6 relative over thousands of steps."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

from parity_helpers import v_app_check, compare, conserved

pytestmark = pytest.mark.gpu

WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def run_pair(ctx, wl, table=None, **kw):
    ref = O.simulate(wl, packets=True, table=table)
    cloud = pdv.Cloud(ctx, wl, table=table)
    try:
        out = pdv.simulate_spectrum(ctx, cloud, wl, precision="fp32", packets=True, **kw)
    finally:
        cloud.close()
    return out, ref


def test_cfg1_paper_layers(ctx):
    wl = W.cfg1(n_packets=20000, n_layers=1000, **WIDE)
    out, ref = run_pair(ctx, wl)
    compare(out, ref, wl, "fp32")
    assert all(conserved(r) for r in out["counters"])
    assert ctx.stats()["last_steps"] > 1000 * wl.n_packets     # every packet crosses the cloud


@pytest.mark.parametrize("kw", [
    dict(n_layers=37),
    dict(n_layers=5000, n_packets=5000),
    dict(n_layers=400, surface_mode=1, reflectivity=1.0),
    dict(n_layers=400, surface_mode=2, reflectivity=0.3),
    dict(n_layers=400, reflectivity=0.0),
    dict(n_layers=400, phase=W.Phase(albedo=1.0), m0=2 * W.MG_CM2),
    dict(n_layers=400, phase=W.Phase(albedo=0.0)),
    dict(n_layers=400, profile_kind="tabulated", prof_v=[2100.0, 2600.0, 3000.0, 4200.0],
         prof_f=[3.0, 1.0, 2.0, 0.2], v_max=0.0, m0=1 * W.MG_CM2),
    dict(n_layers=400, t_snap=(0.5e-6, 1e-6, 1.7e-6, 3e-6)),
    dict(n_layers=400, r_ap=0.0, cone_alpha=2.0),
    dict(n_layers=400, r_ap=0.0, cone_alpha=0.5, t_snap=(1.0e-6, 0.7e-6, 2.0e-6)),
    dict(n_layers=300, max_events=500),
    dict(n_layers=400, phase=W.Phase(kind="mie", m=3.0 + 9.0j, n_angle=1801, n_size=32),
         d_m=1.5e-6, sigma_ln=0.5, m0=2 * W.MG_CM2, v_max=0.0, n_packets=8000),
], ids=["coarse", "fine", "lambert", "specular", "R0", "albedo1", "albedo0", "tabulated",
        "snapshots", "detect_all", "open_aperture_3t", "step_limit", "mie"])
def test_variants(ctx, kw):
    wl = W.cfg1(n_packets=kw.pop("n_packets", 20000), **WIDE).replace(**kw)
    out, ref = run_pair(ctx, wl)
    compare(out, ref, wl, "fp32")
    assert all(conserved(r) for r in out["counters"])


def test_non_uniform_phase_grid(ctx):
    """A phase table on a non-uniform angle grid (binary search in the
    acceptance-rejection lookup)."""
    th = np.pi * np.linspace(0.0, 1.0, 701) ** 1.6
    g = 0.6
    p = (1 - g * g) / (1 + g * g - 2 * g * np.cos(th)) ** 1.5
    wl = W.cfg1(n_packets=20000, n_layers=500,
                phase=W.Phase(kind="table", theta=th, p=p, albedo=0.8, q_ext=2.0), **WIDE)
    out, ref = run_pair(ctx, wl)
    compare(out, ref, wl, "fp32")


def test_runs_are_deterministic_and_ranges_add_up(ctx):
    wl = W.cfg1(n_packets=12000, n_layers=300, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    try:
        a = pdv.simulate_spectrum(ctx, cloud, wl)["raw"]
        b = pdv.simulate_spectrum(ctx, cloud, wl)["raw"]
        assert np.array_equal(a, b)
        lo = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=5000)["raw"]
        hi = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=7000, packet_begin=5000)["raw"]
        assert np.array_equal(lo + hi, a)
    finally:
        cloud.close()


def test_layer_stepping_differs_from_exact_paths_only_by_its_bias(ctx):
    """Same workload, exact free paths vs 2000 layers: different random number
    use, so a statistical comparison of the detected spectra."""
    wl = W.cfg1(n_packets=400000, m0=1.0 * W.MG_CM2, n_bins=60, r_ap=0.0, cone_alpha=2.0)
    cloud = pdv.Cloud(ctx, wl)
    try:
        ex = pdv.simulate_spectrum(ctx, cloud, wl)["raw"][0, 1:-1].astype(np.float64) / 2.0**32
        st = pdv.simulate_spectrum(ctx, cloud, wl.replace(n_layers=2000))["raw"][0, 1:-1]
        st = st.astype(np.float64) / 2.0**32
    finally:
        cloud.close()
    sel = (ex + st) > 50
    z2 = (ex[sel] - st[sel]) ** 2 / (ex[sel] + st[sel])
    assert z2.mean() < 2.0, z2.mean()


def test_invalid_combinations(ctx):
    wl = W.cfg1(n_packets=1000, n_layers=100, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    try:
        with pytest.raises(pdv.PdvError) as e:
            pdv.simulate_spectrum(ctx, cloud, wl, precision="fp64")
        assert e.value.status == pdv.PDV_EINVAL
        req = pdv.Request(cloud, wl)
        with pytest.raises(pdv.PdvError):
            pdv.pdv_simulate_batch(ctx.handle, [req.c])
        with pytest.raises(pdv.PdvError):
            pdv.pdv_submit(ctx.handle, req.c)
        req.c.n_layers = 0
        req.c.reserved = 1
        with pytest.raises(pdv.PdvError):
            pdv.pdv_simulate_spectrum(ctx.handle, req.c)
    finally:
        cloud.close()


def test_full_size_fig4_sampled_packets(ctx):
    """The measured workload (Fig. 4 cloud, 1e7 photons x 1000 layers) in the
    launch bench.py times, with packet records dumped to device memory;
    2000 packets from three places in the range against the oracle."""
    torch = pytest.importorskip("torch")
    wl = W.fig4()
    n = wl.n_packets
    cloud = pdv.Cloud(ctx, wl)
    try:
        dev = {"spectrum": torch.zeros(wl.n_bins, dtype=torch.float64, device="cuda"),
               "raw": torch.zeros(wl.n_bins + 2, dtype=torch.int64, device="cuda"),
               "counters": torch.zeros(len(pdv.COUNTER_NAMES), dtype=torch.int64, device="cuda"),
               "packets": torch.zeros(n * pdv.PACKET_DTYPE.itemsize, dtype=torch.uint8,
                                      device="cuda")}
        req = pdv.Request(cloud, wl, device_out=dev)
        req.c.out_packets = dev["packets"].data_ptr()
        torch.cuda.synchronize()
        pdv.pdv_simulate_spectrum(ctx.handle, req.c)
        torch.cuda.synchronize()
        cnt = dev["counters"].cpu().numpy().astype(np.uint64)
        assert conserved(cnt)
        table = O.phase_table(wl)
        same = tot = 0
        for begin in (0, n // 2, n - 700):
            m = 700 if begin == n - 700 else 650
            g = np.frombuffer(dev["packets"][begin * pdv.PACKET_DTYPE.itemsize:
                                             (begin + m) * pdv.PACKET_DTYPE.itemsize]
                              .cpu().numpy().tobytes(), dtype=pdv.PACKET_DTYPE)
            o = O.simulate(wl, n_packets=m, packet_begin=begin, packets=True, table=table)["packets"]
            eq = g["n_events"] == o["n_events"]
            same += int(eq.sum())
            tot += m
            ok, checked, rep = v_app_check(g, o, wl.v_fs, "fp32")
            assert ok[checked].all(), rep
        assert same / tot >= 0.999, same / tot
    finally:
        cloud.close()
