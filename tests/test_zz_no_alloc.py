"""pdv_simulate_spectrum_static: the spectrum call for code that must not
allocate device memory while it runs.

Some callers cannot call cudaMalloc once they are running: a process whose
device memory is planned up front (every byte assigned at start-up), or one
whose memory belongs to an outside allocator that forbids further
allocations. For them the library offers this entry point, which keeps its
scratch in a fixed 4 MiB device array that the library holds for the life of
the process; the caller still provides the cloud and the output buffers.

The tests run the same requests through this entry point and through
pdv_simulate_spectrum, twice in a row with different sizes (the array keeps
the previous call's contents, which must be cleared), and require identical
integer tallies and spectra, the tolerance every other parity test uses for
integer tallies. The context is made with a counting device allocator, and
the fixed-scratch calls must not call it, nor change the device's free memory.
Requests at the documented size limit are accepted and one step past it are
refused with PDV_EINVAL. The file is self-contained, so it passes in a fresh
process as well as after the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCRATCH = 4 << 20


def scratch_bytes(n_snap, n_bins):
    """The scratch a request needs, as include/pdv.h states it."""
    c = lambda b: (b + 255) // 256 * 256
    return 2048 + c(8 * n_snap * (n_bins + 3)) + c(24 * n_snap)


class CountingAllocator:
    """A pdv_allocator that counts its calls and takes memory from torch's
    caching allocator on the stream the library names."""

    def __init__(self, torch):
        self.calls = 0
        ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
        FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

        def alloc(n, stream, user):
            self.calls += 1
            return torch.cuda.caching_allocator_alloc(int(n), 0, int(stream or 0))

        def free(p, stream, user):
            self.calls += 1
            torch.cuda.caching_allocator_delete(int(p))

        self._cb = (ALLOC(alloc), FREE(free))
        self.c = pdv.pdv_allocator(C.cast(self._cb[0], C.c_void_p), C.cast(self._cb[1], C.c_void_p),
                                   None)


def _device_outputs(torch, wl):
    ns, nb = len(wl.t_snap), wl.n_bins
    return {"spectrum": torch.full((ns * nb,), -1.0, dtype=torch.float64, device="cuda"),
            "raw": torch.full((ns * (nb + 2),), -1, dtype=torch.int64, device="cuda"),
            "counters": torch.full((ns * len(pdv.COUNTER_NAMES),), -1, dtype=torch.int64, device="cuda")}


def _run(ctx, cloud, wl, torch, static, alloc=None):
    out = _device_outputs(torch, wl)
    req = pdv.Request(cloud, wl, device_out=out)
    torch.cuda.synchronize()      # the fills run on torch's stream, not the context's
    if static:
        before = alloc.calls if alloc else 0
        free0 = torch.cuda.mem_get_info()[0]
        pdv.pdv_simulate_spectrum_static(ctx.handle, req.c)
        torch.cuda.synchronize()
        if alloc:
            assert alloc.calls == before, "the fixed-scratch call used the device allocator"
        assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed"
    else:
        pdv.pdv_simulate_spectrum(ctx.handle, req.c)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _same(a, b, wl):
    assert np.array_equal(a["raw"], b["raw"])
    assert np.array_equal(a["counters"], b["counters"])
    assert np.array_equal(a["spectrum"], b["spectrum"])
    assert a["counters"].reshape(-1, len(pdv.COUNTER_NAMES))[0, 0] == wl.n_packets


def test_static_scratch_matches_allocating_call():
    torch = pytest.importorskip("torch")
    alloc = CountingAllocator(torch)
    ctx = pdv.Context(0, allocator=alloc.c)
    try:
        big = W.cfg2(n_packets=400000, t_snap=(1e-6, 2e-6, 3e-6, 4e-6), r_ap=3e-3,
                     cone_alpha=0.5)
        small = W.cfg1(n_packets=300000, r_ap=3e-3, cone_alpha=0.5, n_bins=50)
        clouds = {id(big): pdv.Cloud(ctx, big), id(small): pdv.Cloud(ctx, small)}
        assert alloc.calls > 0            # the clouds' tables came from the allocator
        for wl in (big, small):           # two calls in a row, the second smaller
            cloud = clouds[id(wl)]
            a = _run(ctx, cloud, wl, torch, static=True, alloc=alloc)
            b = _run(ctx, cloud, wl, torch, static=False)
            _same(a, b, wl)
        for c in clouds.values():
            c.close()
    finally:
        ctx.close()


def test_static_scratch_size_limit():
    """At the limit of the 4 MiB array (8 snapshot times, 65497 bins) the call
    runs and equals the allocating call; one bin more is refused."""
    torch = pytest.importorskip("torch")
    ctx = pdv.Context(0)
    try:
        t8 = tuple(np.linspace(1e-6, 4e-6, 8))
        edge = W.cfg1(n_packets=50000, r_ap=3e-3, cone_alpha=0.5, t_snap=t8, n_bins=65497)
        over = edge.replace(n_bins=65498)
        assert scratch_bytes(8, 65497) <= SCRATCH < scratch_bytes(8, 65498)
        cloud = pdv.Cloud(ctx, edge)
        a = _run(ctx, cloud, edge, torch, static=True)
        b = _run(ctx, cloud, edge, torch, static=False)
        _same(a, b, edge)
        req = pdv.Request(cloud, over, device_out=_device_outputs(torch, over))
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_simulate_spectrum_static(ctx.handle, req.c)
        assert e.value.status == pdv.PDV_EINVAL
        cloud.close()
    finally:
        ctx.close()
