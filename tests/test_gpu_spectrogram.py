"""A spectrogram (one request over many snapshot times) equals the
single-snapshot requests at those times, tally for tally (the packets are
transported once and tested at every time; common random numbers)."""
import numpy as np
import pytest

from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import spectrogram as S
from paper_2012_00963_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_rows_equal_single_snapshot_requests():
    ctx = pdv.Context(0)
    try:
        wl = W.cfg2(n_packets=2_000_000, t_snap=(1e-6,), r_ap=3e-3, cone_alpha=0.5)
        cloud = pdv.Cloud(ctx, wl)
        t = np.linspace(0.5e-6, 5e-6, 64)
        sg = S.spectrogram(ctx, cloud, wl, t)
        assert sg["image"].shape == (64, wl.n_bins)
        for i in (0, 17, 40, 63):
            one = pdv.simulate_spectrum(ctx, cloud, wl, snapshots=[t[i]])
            assert np.array_equal(one["raw"][0], sg["raw"][i])
            assert np.array_equal(one["spectrum"][0], sg["image"][i])
        # snapshot order does not matter
        perm = np.random.default_rng(1).permutation(64)
        sp = S.spectrogram(ctx, cloud, wl, t[perm])
        assert np.array_equal(sp["raw"], sg["raw"][perm])
        cloud.close()
    finally:
        ctx.close()
