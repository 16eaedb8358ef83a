"""The request limits of the C ABI at their maximum, against the FP64 oracle
packet by packet (the same bar as tests/test_gpu_parity.py): 4096 snapshot
times with a finite aperture (one histogram row per time, the aperture
interval search over 4096 sorted times) and with an unlimited one (one row
read back for every time), 65536 velocity bins, and one past each limit
refused. The largest per-packet event limit (2^32 - 1, taken as 2^32 - 2)
runs and gives the tallies of the default limit, which no walk here reaches."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

from parity_helpers import compare, conserved

pytestmark = pytest.mark.gpu

MAX_SNAP, MAX_BINS = 4096, 65536
WIDE = dict(r_ap=3e-3, cone_alpha=0.5)


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def run_pair(ctx, wl, precision="fp32"):
    ref = O.simulate(wl, packets=True)
    cloud = pdv.Cloud(ctx, wl)
    try:
        out = pdv.simulate_spectrum(ctx, cloud, wl, precision=precision, packets=True)
    finally:
        cloud.close()
    return out, ref


def times(n):
    # shuffled, so the request order differs from the ascending one; the
    # cloud top (6000 m/s x t) stays below the 50 mm probe plane
    t = np.linspace(0.2e-6, 8.0e-6, n)
    return tuple(np.random.default_rng(5).permutation(t))


@pytest.mark.parametrize("aperture", [WIDE, dict(r_ap=0.0, cone_alpha=0.5)],
                         ids=["finite_aperture", "open_aperture"])
def test_maximum_snapshot_count(ctx, aperture):
    wl = W.cfg1(n_packets=3000, t_snap=times(MAX_SNAP), **aperture)
    out, ref = run_pair(ctx, wl)
    compare(out, ref, wl, "fp32")
    assert all(conserved(r) for r in out["counters"])


def test_maximum_bin_count(ctx):
    wl = W.cfg1(n_packets=20000, n_bins=MAX_BINS, **WIDE)
    out, ref = run_pair(ctx, wl)
    compare(out, ref, wl, "fp32")
    assert out["raw"].shape[1] == MAX_BINS + 2


def test_one_past_each_limit_is_refused(ctx):
    cloud_wl = W.cfg1(n_packets=1000)
    cloud = pdv.Cloud(ctx, cloud_wl)
    try:
        for wl in (cloud_wl.replace(t_snap=times(MAX_SNAP + 1)), cloud_wl.replace(n_bins=MAX_BINS + 1)):
            with pytest.raises(pdv.PdvError) as e:
                pdv.simulate_spectrum(ctx, cloud, wl)
            assert e.value.status == pdv.PDV_EINVAL
    finally:
        cloud.close()


def test_largest_event_limit(ctx):
    wl = W.cfg1(n_packets=20000, **WIDE)
    cloud = pdv.Cloud(ctx, wl)
    try:
        outs = [pdv.simulate_spectrum(ctx, cloud, wl.replace(max_events=m), raw=True)
                for m in (1_000_000, 2**32 - 1)]
    finally:
        cloud.close()
    np.testing.assert_array_equal(outs[0]["raw"], outs[1]["raw"])
    np.testing.assert_array_equal(outs[0]["counters"], outs[1]["counters"])
    assert pdv.counters_dict(outs[1]["counters"][0])["truncated"] == 0
