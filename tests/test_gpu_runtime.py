"""Batched launches (captured-graph persistent kernel over many parameter sets),
the autotuner, and the continuous-batching serving loop: every result equals
the same request run alone, bit for bit (counter-based RNG keyed by the
request's own seed and packet index, integer tallies)."""
import time

import numpy as np
import pytest

from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def small_sets(n, n_max=3e5):
    sets = W.cfg4_sets(n_sets=n, seed=44, n_min=2e4, n_max=n_max)
    # HG phase keeps the set-up cheap; the sets still differ in every cloud parameter
    return [s.replace(phase=W.Phase(kind="hg", g=0.6 + 0.01 * i, albedo=0.5 + 0.02 * i),
                      r_ap=2e-3, cone_alpha=0.4) for i, s in enumerate(sets)]


def test_batch_equals_individual_requests(ctx):
    wls = small_sets(12)
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
    for rep in range(2):   # second call replays the cached graph
        batch = pdv.simulate_batch(ctx, clouds, wls)
        for a, b in zip(alone, batch):
            assert np.array_equal(a["raw"], b["raw"])
            assert np.array_equal(a["counters"], b["counters"])
    for c in clouds:
        c.close()


def test_batch_with_mixed_precision_and_multi_snapshot(ctx):
    wls = small_sets(4)
    wls[1] = wls[1].replace(precision="fp64")
    wls[2] = wls[2].replace(t_snap=(1e-6, 2e-6, 3e-6))
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
    batch = pdv.simulate_batch(ctx, clouds, wls)
    for a, b in zip(alone, batch):
        assert np.array_equal(a["raw"], b["raw"])
    for c in clouds:
        c.close()


@pytest.mark.parametrize("hist_mode", [1, 2])
def test_batch_mixes_open_and_finite_apertures(ctx, hist_mode):
    """Sets with an unlimited aperture tally one histogram row for all their
    snapshot times; in a batch beside aperture-limited sets, and with global
    or privatised histograms, every set equals its run alone."""
    wls = small_sets(4)
    wls[0] = wls[0].replace(r_ap=0.0, t_snap=(1e-6, 2e-6, 3e-6))
    wls[1] = wls[1].replace(r_ap=0.0, cone_alpha=2.0, t_snap=(3e-6, 1e-6))
    wls[2] = wls[2].replace(t_snap=(1e-6, 2.5e-6))
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
    ctx.set_tuning(hist_mode=hist_mode)
    try:
        batch = pdv.simulate_batch(ctx, clouds, wls)
    finally:
        ctx.set_tuning()
    for w, a, b in zip(wls, alone, batch):
        assert np.array_equal(a["raw"], b["raw"])
        assert np.array_equal(a["counters"], b["counters"])
        if w.r_ap <= 0.0:
            assert all(np.array_equal(a["raw"][0], row) for row in a["raw"][1:])
    for c in clouds:
        c.close()


def test_autotune_keeps_results(ctx):
    wls = small_sets(6)
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    before = pdv.simulate_batch(ctx, clouds, wls)
    reqs = [pdv.Request(c, w) for c, w in zip(clouds, wls)]
    t = pdv.pdv_autotune(ctx.handle, [r.c for r in reqs])
    assert t["block_threads"] in (128, 256) and t["hist_mode"] in (1, 2)
    assert t["tile_packets"] in (32, 64, 256) and t["blocks_per_sm"] in (0, 2)
    after = pdv.simulate_batch(ctx, clouds, wls)
    for a, b in zip(before, after):
        assert np.array_equal(a["raw"], b["raw"])
    ctx.set_tuning()   # back to defaults
    for c in clouds:
        c.close()


def test_serving_results_equal_standalone(ctx):
    """Requests submitted while others run are admitted into the running batch
    loop; each one's tallies equal the same request run alone."""
    arrivals = W.cfg5_arrivals(rate=2000.0, duration=0.01, seed=9, n_min=1e4, n_max=2e6)[:16]
    wls = [W.cfg5_request(a, r_ap=2e-3, cone_alpha=0.4) for a in arrivals]
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    alone = [pdv.simulate_spectrum(ctx, c, w) for c, w in zip(clouds, wls)]
    reqs, tickets = [], []
    for c, w in zip(clouds, wls):
        r = pdv.Request(c, w)
        reqs.append(r)
        tickets.append(pdv.pdv_submit(ctx.handle, r.c))
    t0 = time.time()
    pending = set(range(len(tickets)))
    while pending and time.time() - t0 < 120:
        for i in list(pending):
            if pdv.pdv_poll(ctx.handle, tickets[i], 1000) == pdv.PDV_OK:
                pending.discard(i)
    assert not pending
    for a, r in zip(alone, reqs):
        b = r.result()
        assert np.array_equal(a["raw"], b["raw"])
        assert np.array_equal(a["counters"], b["counters"])
    for c in clouds:
        c.close()


def test_serving_cancel_and_unknown_ticket(ctx):
    wl = W.cfg1(n_packets=50_000_000)
    cloud = pdv.Cloud(ctx, wl)
    r = pdv.Request(cloud, wl)
    t = pdv.pdv_submit(ctx.handle, r.c)
    pdv.pdv_cancel(ctx.handle, t)
    with pytest.raises(pdv.PdvError) as e:
        while pdv.pdv_poll(ctx.handle, t, 100000) == pdv.PDV_ENOTREADY:
            pass
    assert e.value.status == pdv.PDV_ECANCELLED
    with pytest.raises(pdv.PdvError) as e:
        pdv.pdv_poll(ctx.handle, 987654321, 0)
    assert e.value.status == pdv.PDV_EINVAL
    # the context still serves new work afterwards
    small = wl.replace(n_packets=10000)
    r2 = pdv.Request(cloud, small)
    t2 = pdv.pdv_submit(ctx.handle, r2.c)
    while pdv.pdv_poll(ctx.handle, t2, 100000) == pdv.PDV_ENOTREADY:
        pass
    ref = pdv.simulate_spectrum(ctx, cloud, small)
    assert np.array_equal(ref["raw"], r2.result()["raw"])
    time.sleep(0.5)
    cloud.close()


def _wait(ctx, t, seconds=60.0):
    t0 = time.time()
    while pdv.pdv_poll(ctx.handle, t, 100000) == pdv.PDV_ENOTREADY:
        assert time.time() - t0 < seconds


def test_admission_by_request_slots(ctx):
    """With one request slot, a second submit is refused with PDV_EAGAIN while
    the first is held (running, or finished and not yet polled), and is
    admitted once the first has been returned by pdv_poll."""
    wl = W.cfg1(n_packets=20_000_000)
    cloud = pdv.Cloud(ctx, wl)
    small = wl.replace(n_packets=20000, seed=77)
    pdv.pdv_set_serving_limits(ctx.handle, 1, 256 << 20)
    try:
        r1, r2 = pdv.Request(cloud, wl), pdv.Request(cloud, small)
        t1 = pdv.pdv_submit(ctx.handle, r1.c)
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_submit(ctx.handle, r2.c)
        assert e.value.status == pdv.PDV_EAGAIN
        _wait(ctx, t1)
        t2 = pdv.pdv_submit(ctx.handle, r2.c)
        _wait(ctx, t2)
        assert np.array_equal(r2.result()["raw"], pdv.simulate_spectrum(ctx, cloud, small)["raw"])
    finally:
        pdv.pdv_set_serving_limits(ctx.handle, 1024, 256 << 20)
        time.sleep(0.2)
        cloud.close()


def test_admission_by_free_device_memory(ctx):
    """A memory reserve larger than the device's free memory refuses every
    submit with PDV_EAGAIN; with the default reserve the same request is
    admitted and runs."""
    torch = pytest.importorskip("torch")
    wl = W.cfg1(n_packets=20000, seed=78)
    cloud = pdv.Cloud(ctx, wl)
    free, total = torch.cuda.mem_get_info()
    try:
        pdv.pdv_set_serving_limits(ctx.handle, 1024, total + (1 << 30))
        r = pdv.Request(cloud, wl)
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_submit(ctx.handle, r.c)
        assert e.value.status == pdv.PDV_EAGAIN
        pdv.pdv_set_serving_limits(ctx.handle, 1024, 256 << 20)
        t = pdv.pdv_submit(ctx.handle, r.c)
        _wait(ctx, t)
        assert np.array_equal(r.result()["raw"], pdv.simulate_spectrum(ctx, cloud, wl)["raw"])
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_set_serving_limits(ctx.handle, 0, 0)
        assert e.value.status == pdv.PDV_EINVAL
    finally:
        pdv.pdv_set_serving_limits(ctx.handle, 1024, 256 << 20)
        time.sleep(0.2)
        cloud.close()


@pytest.mark.parametrize("tile", [16, 32, 256, 1000])
def test_chunk_size_keeps_results(ctx, tile):
    """The packets a warp claims at a time (tile_packets) only schedules work:
    single requests and batches give the same tallies for every value."""
    wls = small_sets(5)
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    ref_one = pdv.simulate_spectrum(ctx, clouds[0], wls[0])
    ref = pdv.simulate_batch(ctx, clouds, wls)
    ctx.set_tuning(tile_packets=tile)
    try:
        one = pdv.simulate_spectrum(ctx, clouds[0], wls[0])
        got = pdv.simulate_batch(ctx, clouds, wls)
    finally:
        ctx.set_tuning()
    assert np.array_equal(one["raw"], ref_one["raw"])
    for a, b in zip(ref, got):
        assert np.array_equal(a["raw"], b["raw"])
        assert np.array_equal(a["counters"], b["counters"])
    for c in clouds:
        c.close()


def test_autotune_cache_round_trip(ctx, tmp_path):
    """With a cache file, the first autotune times the candidates and records
    its choice under the device and batch shape; the next one takes it from the
    file without timing; results stay those of the untuned launch."""
    import json
    wls = small_sets(4)
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    before = pdv.simulate_batch(ctx, clouds, wls)
    reqs = [pdv.Request(c, w) for c, w in zip(clouds, wls)]
    path = str(tmp_path / "tune.json")
    pdv.pdv_set_autotune_cache(ctx.handle, path)
    try:
        t0 = time.perf_counter()
        first = pdv.pdv_autotune(ctx.handle, [r.c for r in reqs])
        t_first = time.perf_counter() - t0
        table = json.load(open(path))
        assert len(table) == 1
        (key, entry), = table.items()
        assert entry["tile_packets"] == first["tile_packets"] in (32, 64, 256)
        ctx.set_tuning()
        t0 = time.perf_counter()
        second = pdv.pdv_autotune(ctx.handle, [r.c for r in reqs])
        t_second = time.perf_counter() - t0
        assert second == first and t_second < 0.2 * t_first
        assert json.load(open(path)) == table
        after = pdv.simulate_batch(ctx, clouds, wls)
        for a, b in zip(before, after):
            assert np.array_equal(a["raw"], b["raw"])
    finally:
        pdv.pdv_set_autotune_cache(ctx.handle, None)
        ctx.set_tuning()
        for c in clouds:
            c.close()
