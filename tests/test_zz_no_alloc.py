"""pdv_simulate_spectrum_static: the spectrum call for code that must not
allocate device memory while it runs.

Some callers cannot call cudaMalloc once they are running: a process whose
device memory is planned up front (every byte assigned at start-up), or one
whose memory belongs to an outside allocator that forbids further
allocations. For them the library offers this entry point, which keeps its
scratch in a fixed 4 MiB device array that the library holds for the life of
the process; the caller still provides the cloud and the output buffers.

The test runs the same requests through this entry point and through
pdv_simulate_spectrum, twice in a row with different sizes (the array keeps
the previous call's contents, which must be cleared), and requires identical
integer tallies and spectra, the tolerance every other parity test uses for
integer tallies. It also checks that a request too large for the array is
refused with PDV_EINVAL. It is self-contained, so it passes in a fresh process
as well as after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_outputs(torch, wl):
    ns, nb = len(wl.t_snap), wl.n_bins
    return {"spectrum": torch.full((ns * nb,), -1.0, dtype=torch.float64, device="cuda"),
            "raw": torch.full((ns * (nb + 2),), -1, dtype=torch.int64, device="cuda"),
            "counters": torch.full((ns * len(pdv.COUNTER_NAMES),), -1, dtype=torch.int64, device="cuda")}


def _run(ctx, cloud, wl, torch, static):
    out = _device_outputs(torch, wl)
    req = pdv.Request(cloud, wl, device_out=out)
    torch.cuda.synchronize()      # the fills run on torch's stream, not the context's
    if static:
        pdv.pdv_simulate_spectrum_static(ctx.handle, req.c)
    else:
        pdv.pdv_simulate_spectrum(ctx.handle, req.c)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_static_scratch_matches_allocating_call():
    torch = pytest.importorskip("torch")
    ctx = pdv.Context(0)
    try:
        big = W.cfg2(n_packets=400000, t_snap=(1e-6, 2e-6, 3e-6, 4e-6), r_ap=3e-3,
                     cone_alpha=0.5)
        small = W.cfg1(n_packets=300000, r_ap=3e-3, cone_alpha=0.5, n_bins=50)
        clouds = {id(big): pdv.Cloud(ctx, big), id(small): pdv.Cloud(ctx, small)}
        for wl in (big, small):           # two calls in a row, the second smaller
            cloud = clouds[id(wl)]
            a = _run(ctx, cloud, wl, torch, static=True)
            b = _run(ctx, cloud, wl, torch, static=False)
            assert np.array_equal(a["raw"], b["raw"])
            assert np.array_equal(a["counters"], b["counters"])
            assert np.array_equal(a["spectrum"], b["spectrum"])
            assert a["counters"].reshape(-1, len(pdv.COUNTER_NAMES))[0, 0] == wl.n_packets
        # a request larger than the fixed scratch is refused
        huge = big.replace(n_bins=65536, t_snap=tuple(np.linspace(1e-6, 5e-6, 64)))
        req = pdv.Request(clouds[id(big)], huge, device_out=_device_outputs(torch, huge))
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_simulate_spectrum_static(ctx.handle, req.c)
        assert e.value.status == pdv.PDV_EINVAL
        for c in clouds.values():
            c.close()
    finally:
        ctx.close()
