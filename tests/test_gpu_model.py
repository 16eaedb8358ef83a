"""GPU parity of the single-scattering spectrum model (pdv_ss_spectrum,
Eq. 22-28) and of the peak extraction (pdv_extract_peaks, Eq. 29-35) against
the FP64 oracle ``oracle/ss_peaks.py``, through the C ABI.

Tolerances (fixed here, from the arithmetic):
* spectrum model: FP32 per bin from FP64 per-set constants; the exponent
  arguments carry about 1e-6 absolute error (x = A0 + D b rounded to FP32 for
  x up to ~20), so each bin is within 1e-5 relative plus 2e-6 of the set's
  largest bin.
* extraction: the DFT sums run over n terms in FP32 with FP32 twiddles
  (2^-24 each); a float32 emulation of the kernel puts the errors of x_peak,
  I''/I, beta and tau0 at or below 2e-6 relative for 600 bins. The test allows
  x_peak 2e-6 absolute (v / v_fs), curvature 5e-5, beta 2.5e-5 and tau0 5e-5
  relative; ten times more for the 8192-bin maximum size (see that test for
  the unsmoothed k_c = n/2 - 1 case, where FP32 input rounding dominates).
* the grid maximum (an argmax over FP32 vs FP64 values) is compared only
  where the oracle's best two window values differ by more than 1e-5
  relative; otherwise any of the tied bins is valid.
"""
import math

import numpy as np
import pytest

from oracle import ss_peaks as O
from paper_2012_00963_gb300 import pdv

pytestmark = pytest.mark.gpu

SETS = [  # beta, tau0, v_fs, v_max (0: untruncated), prefactor
    (5.0, 3.7, 2000.0, 7526.0, 1.0),
    (10.0, 23.4, 2000.0, 0.0, 1.0),
    (3.0, 0.01, 1500.0, 5000.0, 2.5),
    (10.5, 28.79, 2013.0, 0.0, 1.0),
    (2.0, 80.0, 3000.0, 12000.0, 0.3),
    (5.0, 0.0, 2000.0, 6000.0, 1.0),          # tau0 = 0: no signal
    (5.0, 8.0, 2000.0, 6000.0, 1.0),          # v_fs (2000) and v_max (6000) on bin edges
    (5.0, 8.0, 2000.0, 2005.0, 1.0),          # the whole support inside one bin
    (5.0, 8.0, 9000.0, 0.0, 1.0),             # support above the range
    (7.0, 15.0, 1000.0, 0.0, 1.0),            # v_fs below the range start (v_lo = 1500 case)
]


@pytest.fixture(scope="module")
def ctx():
    c = pdv.Context(0)
    yield c
    c.close()


def oracle_bins(p, n_bins, v_lo, v_hi, per_dv=False):
    beta, tau0, v_fs, v_max, pref = p
    vm = v_max if (v_max > v_fs and math.isfinite(v_max)) else math.inf
    return O.ss_spectrum_bins(beta, tau0, v_fs, n_bins, v_lo, v_hi, v_max=vm, prefactor=pref,
                              per_dv=per_dv)


def assert_bins_close(g, o):
    scale = np.max(np.abs(o)) if o.size else 0.0
    err = np.abs(g - o)
    assert np.all(err <= 1e-5 * np.abs(o) + 2e-6 * scale), float(np.max(err - 1e-5 * np.abs(o)))


@pytest.mark.parametrize("n_bins,v_lo,v_hi,per_dv", [
    (600, 0.0, 8000.0, False), (600, 0.0, 8000.0, True), (1001, 1500.0, 9000.0, False),
    (7, 0.0, 8000.0, False), (1, 0.0, 8000.0, True)])
def test_ss_spectrum_matches_oracle(ctx, n_bins, v_lo, v_hi, per_dv):
    g = pdv.ss_spectrum(ctx, SETS, n_bins, v_lo, v_hi, per_dv=per_dv)
    for i, p in enumerate(SETS):
        assert_bins_close(g[i], oracle_bins(p, n_bins, v_lo, v_hi, per_dv))


def test_ss_spectrum_total_and_zero_cases(ctx):
    g = pdv.ss_spectrum(ctx, SETS, 600, 0.0, 8000.0)
    # truncated laws inside the range integrate to P (1 - exp(-tau0))
    for i in (0, 6, 7):
        b, t, vf, vm, P = SETS[i]
        assert g[i].sum() == pytest.approx(P * -math.expm1(-t), rel=2e-5)
    assert np.all(g[5] == 0.0)            # tau0 = 0
    assert np.all(g[8] == 0.0)            # support above the range
    assert np.all(g[0, :150] == 0.0)      # below v_fs


def test_ss_spectrum_device_buffers_and_invalid_sets(ctx):
    torch = pytest.importorskip("torch")
    arr = np.array(SETS, dtype=np.float64)
    host = pdv.ss_spectrum(ctx, SETS, 600, 0.0, 8000.0)
    d_sets = torch.tensor(arr, device="cuda")
    d_out = torch.full((len(SETS) * 600,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    pdv.pdv_ss_spectrum(ctx.handle, d_sets, len(SETS), 600, 0.0, 8000.0, d_out)
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy().reshape(len(SETS), 600), host)
    # host-side validation
    bad = np.zeros(1, dtype=pdv.SS_SET_DTYPE)
    bad[0] = (0.0, 1.0, 2000.0, 0.0, 1.0)
    with pytest.raises(pdv.PdvError) as e:
        pdv.pdv_ss_spectrum(ctx.handle, bad, 1, 10, 0.0, 8000.0, np.zeros(10))
    assert e.value.status == pdv.PDV_EINVAL
    # device-side validation: the bad set's bins are NaN, the others are computed
    arr2 = arr.copy()
    arr2[3, 0] = -1.0
    d_sets = torch.tensor(arr2, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(pdv.PdvError) as e:
        pdv.pdv_ss_spectrum(ctx.handle, d_sets, len(SETS), 600, 0.0, 8000.0, d_out)
    assert e.value.status == pdv.PDV_EINVAL
    torch.cuda.synchronize()
    g = d_out.cpu().numpy().reshape(len(SETS), 600)
    assert np.all(np.isnan(g[3]))
    assert np.array_equal(g[[0, 1, 2, 4]], host[[0, 1, 2, 4]])
    with pytest.raises(pdv.PdvError):
        pdv.pdv_ss_spectrum(ctx.handle, arr.view(pdv.SS_SET_DTYPE).ravel(), len(SETS), 0, 0.0,
                            1.0, np.zeros(1))
    pdv.pdv_ss_spectrum(ctx.handle, arr.view(pdv.SS_SET_DTYPE).ravel(), 0, 600, 0.0, 8000.0,
                        np.zeros(1))   # empty batch is a no-op


# ------------------------------------------------------------------ extraction
def gamma_like(n, j0, width, rng, noise):
    """A seeded peaked shape with multiplicative noise (input generator only)."""
    j = np.arange(n, dtype=np.float64)
    z = np.clip((j - j0 + 3 * width) / width, 0.0, None)
    s = z ** 3 * np.exp(-z)
    return s * (1.0 + noise * rng.standard_normal(n))


def extraction_cases(n=600):
    rng = np.random.default_rng(12)
    out = []
    for beta, tau0 in [(10.0, 23.4), (6.0, 8.6), (10.5, 28.79), (4.0, 12.0), (8.0, 40.0)]:
        s = O.ss_spectrum_bins(beta, tau0, 2000.0, n, 0.0, 8000.0, per_dv=True)
        out.append(s)
        out.append(s * (1.0 + 0.03 * rng.standard_normal(n)))
    for j0 in (180.3, 260.0, 333.7):
        out.append(gamma_like(n, j0, 12.0, rng, 0.02))
    return np.array(out)


def compare_peak(g, o, scale=1.0):
    assert int(g["status"]) == o["status"]
    if o["status"] in (O.STATUS_OK, O.STATUS_NOT_MAX):
        assert g["x_peak"] == pytest.approx(o["x_peak"], abs=2e-6 * scale)
        assert g["curvature"] == pytest.approx(o["curvature"], rel=5e-5 * scale)
        assert g["i_peak"] == pytest.approx(o["i_peak"], rel=2e-5 * scale)
    if o["status"] == O.STATUS_OK:
        assert g["beta"] == pytest.approx(o["beta"], rel=2.5e-5 * scale)
        assert g["tau0"] == pytest.approx(o["tau0"], rel=5e-5 * scale)
    else:
        assert math.isnan(g["beta"]) and math.isnan(g["tau0"])


def check_jmax(g, o, s, k_c, lo, hi):
    if o["j_max"] < 0:
        assert int(g["j_max"]) == -1
        return
    sm = O.lowpass(s, k_c)[lo:hi + 1]
    top = np.sort(sm)[-2:] if sm.size > 1 else np.array([-np.inf, sm[0]])
    if top[1] - top[0] > 1e-5 * abs(top[1]):
        assert int(g["j_max"]) == o["j_max"]
    else:
        assert abs(int(g["j_max"]) - o["j_max"]) <= 1


# both products on the tensor cores (split TF32; the default for cut-offs up
# to 63 modes) and as FP32 FMAs on the CUDA cores (PDV_EXTRACT_SIMT)
PATHS = pytest.mark.parametrize("simt", [False, True], ids=["tensor", "simt"])


@PATHS
@pytest.mark.parametrize("k_c,x_min,x_max", [(40, 1.02, 3.5), (60, -math.inf, math.inf),
                                             (25, 1.1, 2.2), (71, 1.02, 3.5), (80, 1.02, 3.5)])
def test_extract_matches_oracle(ctx, k_c, x_min, x_max, simt):
    spec = extraction_cases()
    g = pdv.extract_peaks(ctx, spec, 0.0, 8000.0, 2000.0, k_c, x_min, x_max, simt=simt)
    xc = (0.0 + (np.arange(600) + 0.5) * (8000.0 / 600)) / 2000.0
    lo = int(np.searchsorted(xc, x_min)) if math.isfinite(x_min) else 0
    hi = int(np.searchsorted(xc, x_max, side="right")) - 1 if math.isfinite(x_max) else 599
    for i, s in enumerate(spec):
        o = O.extract_peak(s, 0.0, 8000.0, 2000.0, k_c,
                           x_min if math.isfinite(x_min) else None,
                           x_max if math.isfinite(x_max) else None)
        compare_peak(g[i], o)
        check_jmax(g[i], o, s, k_c, lo, hi)


@PATHS
def test_extract_status_and_edge_cases(ctx, simt):
    n = 300
    cases = [np.zeros(n),                                                  # no peak
             1.0 + np.cos(2 * math.pi * (np.arange(n) - 50) / n),          # falls over the window
             -np.ones(n)]                                                  # negative
    g = pdv.extract_peaks(ctx, np.array(cases), 0.0, 6000.0, 2000.0, 4, 1.2, 2.0, simt=simt)
    for i, s in enumerate(cases):
        o = O.extract_peak(s, 0.0, 6000.0, 2000.0, 4, 1.2, 2.0)
        compare_peak(g[i], o)
        if i < 2:   # unique maxima (the constant case has FP32-rounding ties)
            assert int(g[i]["j_max"]) == o["j_max"]
    assert [int(x) for x in g["status"]] == [pdv.PDV_PEAK_NO_PEAK, pdv.PDV_PEAK_EDGE,
                                            pdv.PDV_PEAK_NO_PEAK]
    # empty window
    g = pdv.extract_peaks(ctx, np.array(cases[1:2]), 0.0, 6000.0, 2000.0, 4, 5.0, 4.0, simt=simt)
    assert int(g[0]["status"]) == pdv.PDV_PEAK_NO_PEAK and int(g[0]["j_max"]) == -1
    # smallest size: 3 bins, one mode
    s = np.array([0.2, 1.0, 0.3])
    g = pdv.extract_peaks(ctx, s, 0.0, 3.0, 1.0, 1, simt=simt)
    compare_peak(g[0], O.extract_peak(s, 0.0, 3.0, 1.0, 1))
    # invalid arguments
    for kw in (dict(k_c=0), dict(k_c=150)):
        with pytest.raises(pdv.PdvError) as e:
            pdv.extract_peaks(ctx, np.ones((1, n)), 0.0, 6000.0, 2000.0, **kw)
        assert e.value.status == pdv.PDV_EINVAL
    with pytest.raises(pdv.PdvError):
        pdv.extract_peaks(ctx, np.ones((1, 8193)), 0.0, 6000.0, 2000.0, 10)
    with pytest.raises(pdv.PdvError):
        pdv.extract_peaks(ctx, np.ones((1, 100)), 0.0, 6000.0, -1.0, 10)


@PATHS
def test_extract_ragged_batches_and_device_buffers(ctx, simt):
    torch = pytest.importorskip("torch")
    base = extraction_cases()
    rng = np.random.default_rng(3)
    big = base[rng.integers(0, len(base), 2000)] * (1.0 + 0.01 * rng.standard_normal((2000, 600)))
    g = pdv.extract_peaks(ctx, big, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5, simt=simt)
    for i in rng.choice(2000, 40, replace=False):
        compare_peak(g[i], O.extract_peak(big[i], 0.0, 8000.0, 2000.0, 40, 1.02, 3.5))
    # a tile's other spectra do not change a spectrum's result: alone, at a
    # ragged tail, and as the last of a full tile
    for lo, hi in ((0, 1), (1990, 2000), (1873, 2000)):
        part = pdv.extract_peaks(ctx, big[lo:hi], 0.0, 8000.0, 2000.0, 40, 1.02, 3.5, simt=simt)
        assert part.tobytes() == g[lo:hi].tobytes()
    d_in = torch.tensor(big, device="cuda")
    d_out = torch.zeros(2000 * pdv.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    pdv.pdv_extract_peaks(ctx.handle, d_in, 2000, 600, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5, d_out,
                          simt=simt)
    torch.cuda.synchronize()
    assert d_out.cpu().numpy().tobytes() == g.tobytes()


@PATHS
def test_extract_unaligned_rows(ctx, simt):
    """Rows that do not start on 16-byte boundaries take the 8-byte loads: a
    device buffer one double past an aligned base gives the same bytes as the
    aligned one, and an odd bin count (601) over several tiles meets the oracle."""
    torch = pytest.importorskip("torch")
    base = extraction_cases()
    rng = np.random.default_rng(5)
    big = base[rng.integers(0, len(base), 300)] * (1.0 + 0.01 * rng.standard_normal((300, 600)))
    d_al = torch.tensor(big, device="cuda")
    d_off = torch.zeros(big.size + 1, dtype=torch.float64, device="cuda")
    d_off[1:] = d_al.view(-1)
    outs = []
    for d_in in (d_al, d_off[1:]):
        d_out = torch.zeros(300 * pdv.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        pdv.pdv_extract_peaks(ctx.handle, d_in, 300, 600, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5,
                              d_out, simt=simt)
        torch.cuda.synchronize()
        outs.append(d_out.cpu().numpy().tobytes())
    assert outs[0] == outs[1]
    odd = np.concatenate([big, big[:, -1:]], axis=1)               # 601 bins, same width
    v_hi = 8000.0 * 601 / 600
    g = pdv.extract_peaks(ctx, odd, 0.0, v_hi, 2000.0, 40, 1.02, 3.5, simt=simt)
    for i in rng.choice(300, 30, replace=False):
        compare_peak(g[i], O.extract_peak(odd[i], 0.0, v_hi, 2000.0, 40, 1.02, 3.5))


def test_extract_paths_agree(ctx):
    """The tensor-core and the CUDA-core products give the same peaks within
    twice the oracle bar (each path is held to 2.5e-5 in beta and 5e-5 in tau0
    against the oracle) on 2000 noisy spectra."""
    base = extraction_cases()
    rng = np.random.default_rng(4)
    big = base[rng.integers(0, len(base), 2000)] * (1.0 + 0.01 * rng.standard_normal((2000, 600)))
    a = pdv.extract_peaks(ctx, big, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5)
    b = pdv.extract_peaks(ctx, big, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5, simt=True)
    ok = a["status"] == pdv.PDV_PEAK_OK
    assert np.array_equal(a["status"], b["status"]) and ok.mean() > 0.5
    assert np.max(np.abs(a["x_peak"][ok] - b["x_peak"][ok])) < 4e-6
    assert np.max(np.abs(a["beta"][ok] / b["beta"][ok] - 1.0)) < 5e-5
    assert np.max(np.abs(a["tau0"][ok] / b["tau0"][ok] - 1.0)) < 1e-4


def test_extract_maximum_size(ctx):
    """8192 bins. With every mode kept (k_c = 4095) nothing is smoothed: the
    rounding of the input to FP32 (6e-8 relative per bin) reaches the second
    derivative amplified by up to pi^2 per bin, against a curvature of
    s / 150^2 for this peak, i.e. one to a few percent relative. That case is
    held to a 5 % curvature bound and 1e-4 in x_peak; a smoothing cut-off (k_c = 64)
    keeps ten times the base tolerance."""
    n = 8192
    rng = np.random.default_rng(5)
    s = gamma_like(n, 3000.5, 150.0, rng, 0.0)
    g = pdv.extract_peaks(ctx, s, 0.0, 8192.0, 2000.0, 4095)[0]
    o = O.extract_peak(s, 0.0, 8192.0, 2000.0, 4095)
    assert int(g["status"]) == o["status"] == O.STATUS_OK
    assert abs(int(g["j_max"]) - o["j_max"]) <= 1     # the peak sits half-way between bins
    assert g["x_peak"] == pytest.approx(o["x_peak"], abs=1e-4)
    assert g["curvature"] == pytest.approx(o["curvature"], rel=5e-2)
    for simt in (False, True):
        g = pdv.extract_peaks(ctx, s, 0.0, 8192.0, 2000.0, 64, simt=simt)
        compare_peak(g[0], O.extract_peak(s, 0.0, 8192.0, 2000.0, 64), scale=10.0)


def test_extract_recovers_model_parameters_on_gpu(ctx):
    """End to end on the GPU: Eq. 28 spectra from pdv_ss_spectrum, then
    pdv_extract_peaks recovers beta and tau0 (the bias left is the oracle's,
    pinned in the oracle tests)."""
    params = [(10.0, 23.4, 2000.0, 0.0, 1.0), (10.5, 28.79, 2013.0, 0.0, 1.0),
              (6.0, 8.6, 2000.0, 0.0, 1.0)]
    spec = pdv.ss_spectrum(ctx, params, 1200, 0.0, 8000.0, per_dv=True)
    for p, s in zip(params, spec):
        g = pdv.extract_peaks(ctx, s, 0.0, 8000.0, p[2], 60, 1.02, 3.5)[0]
        assert int(g["status"]) == pdv.PDV_PEAK_OK
        assert g["beta"] == pytest.approx(p[0], rel=5e-3)
        assert g["tau0"] == pytest.approx(p[1], rel=1.5e-2)


def test_bench_size_sampled():
    """At the measured size (1e5 sets / spectra of 600 bins, the launch
    configuration bench.py times), sampled outputs against the oracle one by
    one. The extraction inputs come from a seeded generator, not from the
    CUDA path."""
    torch = pytest.importorskip("torch")
    from paper_2012_00963_gb300 import workloads as W
    ctx = pdv.Context(0)
    try:
        n, nb = 100_000, 600
        sets = W.model_sets(n)
        d_sets = torch.tensor(sets, device="cuda")
        d_out = torch.empty(n * nb, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pdv.pdv_ss_spectrum(ctx.handle, d_sets, n, nb, 0.0, 8000.0, d_out, per_dv=True)
        torch.cuda.synchronize()
        rng = np.random.default_rng(8)
        for i in rng.choice(n, 12, replace=False):
            b, t, vf, vm, P = sets[i]
            g = d_out[i * nb:(i + 1) * nb].cpu().numpy()
            assert_bins_close(g, O.ss_spectrum_bins(b, t, vf, nb, 0.0, 8000.0, prefactor=P,
                                                    per_dv=True))
        j0 = rng.uniform(170.0, 330.0, n)
        width = rng.uniform(8.0, 25.0, n)
        jj = np.arange(nb)[None, :]
        z = np.clip((jj - j0[:, None] + 3 * width[:, None]) / width[:, None], 0.0, None)
        spec = z ** 3 * np.exp(-z) * (1.0 + 0.02 * rng.standard_normal((n, nb)))
        d_in = torch.tensor(spec, device="cuda")
        d_pk = torch.zeros(n * pdv.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        sample = rng.choice(n, 40, replace=False)
        for simt in (False, True):
            pdv.pdv_extract_peaks(ctx.handle, d_in, n, nb, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5, d_pk,
                                  simt=simt)
            torch.cuda.synchronize()
            got = np.frombuffer(d_pk.cpu().numpy().tobytes(), dtype=pdv.PEAK_DTYPE)
            for i in sample:
                compare_peak(got[i], O.extract_peak(spec[i], 0.0, 8000.0, 2000.0, 40, 1.02, 3.5))
    finally:
        ctx.close()
