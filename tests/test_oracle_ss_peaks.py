"""Pins of the single-scattering model and peak-extraction oracle
(``oracle/ss_peaks.py``) against what the paper and the mathematics fix:
the worked numbers of Section III.C, the closed forms of Eq. 31 and Eq. 34,
the antiderivative of Eq. 28, the optically thin limit, and a pure cosine
spectrum whose peak and curvature are known exactly."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ss_peaks as O

HERE = os.path.dirname(os.path.abspath(__file__))


def test_worked_example_section_iii_c():
    g = json.load(open(os.path.join(HERE, "golden", "peak_worked_example.json")))
    beta, tau0 = O.params_from_peak(g["x_peak"], g["curvature"])
    assert beta == pytest.approx(math.sqrt(110.0), rel=1e-15)
    assert round(beta, 1) == g["beta_printed"]
    # the paper evaluates tau0 with the rounded beta
    assert round(math.exp(g["beta_printed"] * (g["x_peak"] - 1.0)), 2) == g["tau0_printed"]
    assert tau0 == pytest.approx(math.exp(math.sqrt(110.0) * 0.32), rel=1e-15)
    assert math.isnan(O.params_from_peak(1.3, 5.0)[0])


@pytest.mark.parametrize("beta,tau0", [(5.0, 3.7), (10.0, 23.4), (10.5, 28.79), (3.0, 8.6)])
def test_ss_peak_matches_eq31_eq34(beta, tau0):
    """Maximise Eq. 28 numerically (untruncated law) and difference it: the
    maximum sits at Eq. 31 and I''/I there is -beta^2 (Eq. 34)."""
    v_fs = 2000.0
    x = np.linspace(1.0, 1.0 + 3.0 * math.log(max(tau0, 2.0)) / beta + 0.5, 200001)
    i = O.ss_intensity(x * v_fs, beta, tau0, v_fs)
    k = int(np.argmax(i))
    lo, hi = x[k - 1], x[k + 1]
    for _ in range(200):          # golden-section refinement
        m1, m2 = lo + 0.382 * (hi - lo), hi - 0.382 * (hi - lo)
        if O.ss_intensity(m1 * v_fs, beta, tau0, v_fs) > O.ss_intensity(m2 * v_fs, beta, tau0, v_fs):
            hi = m2
        else:
            lo = m1
    xp = 0.5 * (lo + hi)
    x_th, c_th = O.ss_peak_theory(beta, tau0)
    assert xp == pytest.approx(x_th, abs=1e-7)
    h = 1e-4
    f = lambda y: float(O.ss_intensity(y * v_fs, beta, tau0, v_fs))
    curv = (f(x_th + h) - 2.0 * f(x_th) + f(x_th - h)) / (h * h) / f(x_th)
    assert curv == pytest.approx(c_th, rel=1e-5)


@pytest.mark.parametrize("tau0", [0.3, 3.7, 23.4, 80.0])
def test_ss_bins_integrate_to_one_minus_exp(tau0):
    """tau0 f exp(-tau0 Fbar) is the derivative of exp(-tau0 Fbar), and Fbar
    runs from 1 at v_fs to 0 at v_max: the bins sum to P (1 - exp(-tau0))."""
    beta, v_fs, v_max = 5.0, 2000.0, 7526.0
    s = O.ss_spectrum_bins(beta, tau0, v_fs, 600, 0.0, 8000.0, v_max=v_max, prefactor=2.5)
    assert s.sum() == pytest.approx(2.5 * -math.expm1(-tau0), rel=1e-12)
    assert np.all(s[:150] == 0.0) and np.all(s[565:] == 0.0)   # outside [v_fs, v_max]
    # untruncated law over a range that holds all but exp(-40) of the mass
    s = O.ss_spectrum_bins(beta, tau0, v_fs, 2000, 0.0, 2000.0 * 9.0, prefactor=1.0)
    assert s.sum() == pytest.approx(-math.expm1(-tau0), rel=1e-12)
    # one bin holding the whole support (the integrand's peak is resolved)
    one = O.ss_spectrum_bins(10.0, tau0, v_fs, 1, 0.0, 8000.0, v_max=v_max)
    assert one[0] == pytest.approx(-math.expm1(-tau0), rel=1e-12)
    # per_dv divides by the bin width
    d = O.ss_spectrum_bins(beta, tau0, v_fs, 2000, 0.0, 18000.0, per_dv=True)
    assert np.allclose(d * 9.0, s, rtol=1e-14, atol=0)


def test_ss_thin_limit_is_the_mass_histogram():
    """tau0 -> 0: the spectrum per unit tau0 is the mass per bin, the integral
    of Eq. 20 over the bin."""
    beta, v_fs, v_max, tau0 = 5.0, 2000.0, 6000.0, 1e-7
    edges = np.linspace(0.0, 8000.0, 201)
    s = O.ss_spectrum_bins(beta, tau0, v_fs, 200, 0.0, 8000.0, v_max=v_max) / tau0
    lo, hi = np.clip(edges[:-1], v_fs, v_max), np.clip(edges[1:], v_fs, v_max)
    e = lambda v: np.exp(-beta * (v / v_fs - 1.0))
    mass = (e(lo) - e(hi)) / (1.0 - math.exp(-beta * (v_max / v_fs - 1.0)))
    assert np.allclose(s, mass, rtol=1e-6, atol=1e-12)


def test_lowpass_keeps_band_limited_signal():
    n = 600
    j = np.arange(n)
    s = 1.0 + 0.3 * np.cos(2 * math.pi * 3 * j / n + 0.2) + 0.1 * np.sin(2 * math.pi * 17 * j / n)
    assert np.allclose(O.lowpass(s, 17), s, atol=1e-13)
    assert not np.allclose(O.lowpass(s, 16), s, atol=1e-3)
    a, b = O.lowpass_coefficients(s, 20)
    for u in (12.0, 100.25, 333.7):
        s0, s1, s2 = O.smooth_derivatives(a, b, n, u)
        ph = 2 * math.pi * 3 * u / n + 0.2
        w3, w17 = 2 * math.pi * 3 / n, 2 * math.pi * 17 / n
        assert s0 == pytest.approx(1.0 + 0.3 * math.cos(ph) + 0.1 * math.sin(w17 * u), abs=1e-12)
        assert s1 == pytest.approx(-0.3 * w3 * math.sin(ph) + 0.1 * w17 * math.cos(w17 * u), abs=1e-12)
        assert s2 == pytest.approx(-0.3 * w3 ** 2 * math.cos(ph) - 0.1 * w17 ** 2 * math.sin(w17 * u),
                                   abs=1e-12)


@pytest.mark.parametrize("j0,m", [(211.37, 2), (250.0, 1), (180.8, 3)])
def test_extract_cosine_peak_exactly(j0, m):
    """s_j = A + B cos(2 pi m (j - j0) / n): the low-pass keeps it, its maximum
    is at bin j0 and I''/I there is -B w^2 / (A + B) in bin units."""
    n, A, B, v_lo, v_hi, v_fs = 600, 0.4, 1.0, 0.0, 8000.0, 2000.0
    dv = (v_hi - v_lo) / n
    j = np.arange(n)
    s = A + B * np.cos(2 * math.pi * m * (j - j0) / n)
    r = O.extract_peak(s, v_lo, v_hi, v_fs, k_c=8, x_min=1.2, x_max=3.0)
    assert r["status"] == O.STATUS_OK
    assert r["x_peak"] == pytest.approx((v_lo + (j0 + 0.5) * dv) / v_fs, abs=1e-12)
    w = 2 * math.pi * m / n
    assert r["curvature"] == pytest.approx(-B * w * w / (A + B) * (v_fs / dv) ** 2, rel=1e-10)
    assert r["i_peak"] == pytest.approx(A + B, rel=1e-12)


@pytest.mark.parametrize("beta,tau0", [(10.0, 23.4), (6.0, 8.6), (10.5, 28.79)])
def test_extract_recovers_eq28_parameters(beta, tau0):
    """Extraction applied to the noise-free Eq. 28 spectrum recovers beta and
    tau0; what is left is the bias of binning and of the low-pass filter. The
    spectrum jumps at v_fs by tau0 (beta / v_fs) exp(-tau0), and the filter
    turns that jump into ringing whose second derivative grows as k_c^2: the
    cut-off keeps the peak's band (about n / (peak width in bins) modes) and
    little more. For optically thin clouds (tau0 of a few) the jump is a
    sizeable part of the peak and the extraction is biased; the paper's cases
    are tau0 = 8.6 to 29."""
    v_fs, n = 2000.0, 1200
    s = O.ss_spectrum_bins(beta, tau0, v_fs, n, 0.0, 8000.0, per_dv=True)
    r = O.extract_peak(s, 0.0, 8000.0, v_fs, k_c=60, x_min=1.02, x_max=3.5)
    assert r["status"] == O.STATUS_OK
    x_th, c_th = O.ss_peak_theory(beta, tau0)
    assert r["x_peak"] == pytest.approx(x_th, abs=1e-3)
    assert r["beta"] == pytest.approx(beta, rel=5e-3)
    assert r["tau0"] == pytest.approx(tau0, rel=1.5e-2)


def test_extract_status_cases():
    n = 300
    r = O.extract_peak(np.zeros(n), 0.0, 6000.0, 2000.0, k_c=20)
    assert r["status"] == O.STATUS_NO_PEAK and math.isnan(r["beta"])
    decreasing = 1.0 + np.cos(2 * math.pi * (np.arange(n) - 50) / n)   # falls over j = 50..200
    r = O.extract_peak(decreasing, 0.0, 6000.0, 2000.0, k_c=4, x_min=1.2, x_max=2.0)
    assert r["status"] == O.STATUS_EDGE
    r = O.extract_peak(np.ones(n), 0.0, 6000.0, 2000.0, k_c=5, x_min=5.0, x_max=4.0)
    assert r["status"] == O.STATUS_NO_PEAK
