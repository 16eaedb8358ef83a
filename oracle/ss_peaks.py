"""FP64 oracle for the single-scattering spectrum model and the peak-based
parameter extraction (Shi et al., arXiv:2012.00963, Section III.B-C).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg use this module. It imports nothing
from the product package and shares no code with the CUDA path.

Single-scattering model (Eq. 22-28). Light is scattered once, straight back,
by particles moving at the velocity v read off the Doppler shift; on the way in
and out it is attenuated by the particles above that layer. With the mass
density f(v) of Eq. 20 normalised to unit area mass and Fbar(v) the fraction of
the mass above v, the amplitude spectrum is, up to a constant,

    I(v) = P tau0 f(v) exp(-tau0 Fbar(v)),

where tau0 is the optical thickness seen by back-scattering and absorption
only (Eq. 25, Eq. 27) and P gathers the size factors of Eq. 28. For the
untruncated exponential law Fbar = (v_fs / beta) f, which is Eq. 28 itself.
When the law is cut at v_max (the clouds the Monte Carlo transports), f and
Fbar are renormalised over [v_fs, v_max].

Peak extraction (Eq. 29-35 and Section III.C). The spectrum is smoothed by an
FFT low-pass filter; the main peak is located, the relative curvature
I''/I there is taken in the velocity variable x = v / v_fs, and

    beta = sqrt(-I''/I)          (Eq. 34, Eq. 35)
    tau0 = exp(beta (x_peak - 1))  (Eq. 31, Eq. 35).

Readings where the paper leaves the procedure open:
* the low-pass filter keeps the Fourier modes 0..k_c of the real DFT of the
  binned spectrum and drops the rest (no window, no padding);
* the smoothed spectrum is the trigonometric polynomial those modes define, so
  its derivatives are taken analytically;
* the peak is the largest smoothed value on the bin centres inside the search
  window, refined by Newton steps on the first derivative (at most
  ``NEWTON_STEPS``, each kept within one bin of the grid maximum).
"""
from __future__ import annotations

import math

import numpy as np

NEWTON_STEPS = 8

STATUS_OK = 0
STATUS_NO_PEAK = 1        # the smoothed maximum in the window is not positive
STATUS_NOT_MAX = 2        # the curvature at the maximum is not negative
STATUS_EDGE = 3           # the maximum sits on an end of the search window


# ------------------------------------------------------------------ Eq. 20
def mass_density(v, beta, v_fs, v_max=math.inf):
    """f(v) of Eq. 20, zero below v_fs; renormalised over [v_fs, v_max] when
    v_max is finite (the cut law of the transported clouds)."""
    v = np.asarray(v, dtype=np.float64)
    f = (beta / v_fs) * np.exp(-beta * (v / v_fs - 1.0))
    if math.isfinite(v_max):
        f = f / (1.0 - math.exp(-beta * (v_max / v_fs - 1.0)))
        f = np.where(v > v_max, 0.0, f)
    return np.where(v < v_fs, 0.0, f)


def mass_above(v, beta, v_fs, v_max=math.inf):
    """Fbar(v): the fraction of the area mass moving faster than v."""
    v = np.asarray(v, dtype=np.float64)
    vv = np.clip(v, v_fs, v_max)
    e = np.exp(-beta * (vv / v_fs - 1.0))
    if math.isfinite(v_max):
        tail = math.exp(-beta * (v_max / v_fs - 1.0))
        return (e - tail) / (1.0 - tail)
    return e


def ss_intensity(v, beta, tau0, v_fs, v_max=math.inf, prefactor=1.0):
    """Eq. 28 at velocity v: P tau0 f(v) exp(-tau0 Fbar(v))."""
    return prefactor * tau0 * mass_density(v, beta, v_fs, v_max) * np.exp(
        -tau0 * mass_above(v, beta, v_fs, v_max))


def ss_spectrum_bins(beta, tau0, v_fs, n_bins, v_lo, v_hi, v_max=math.inf, prefactor=1.0,
                     per_dv=False, n_gauss=16):
    """The single-scattering spectrum integrated over each of ``n_bins``
    uniform bins of [v_lo, v_hi]: composite Gauss-Legendre quadrature of
    Eq. 28 on the part of each bin inside the support [v_fs, v_max] (split
    there, because the integrand jumps at both ends). The integrand varies on
    the scale v_fs / beta (exp(-tau0 Fbar) changes by O(1) per unit of
    beta (v / v_fs - 1)), so each piece is cut into panels no wider than
    v_fs / (8 beta). With ``per_dv`` each bin is divided by its width."""
    xg, wg = np.polynomial.legendre.leggauss(n_gauss)
    edges = v_lo + (v_hi - v_lo) * np.arange(n_bins + 1, dtype=np.float64) / n_bins
    panel = v_fs / (8.0 * beta)
    out = np.zeros(n_bins)
    for b in range(n_bins):
        a, c = max(edges[b], v_fs), min(edges[b + 1], v_max)
        if c <= a:
            continue
        m = max(1, int(math.ceil((c - a) / panel)))
        p = a + (c - a) * np.arange(m + 1, dtype=np.float64) / m
        total = 0.0
        for i in range(m):
            v = 0.5 * (p[i + 1] - p[i]) * xg + 0.5 * (p[i + 1] + p[i])
            total += 0.5 * (p[i + 1] - p[i]) * np.sum(
                wg * ss_intensity(v, beta, tau0, v_fs, v_max, prefactor))
        out[b] = total
    if per_dv:
        out /= (v_hi - v_lo) / n_bins
    return out


def ss_peak_theory(beta, tau0):
    """Eq. 31 and Eq. 34: peak position x_peak = 1 + ln(tau0) / beta and
    relative curvature -beta^2 (in x = v / v_fs) of the untruncated model."""
    return 1.0 + math.log(tau0) / beta, -beta * beta


# ------------------------------------------------------------------ Eq. 35
def params_from_peak(x_peak, curvature):
    """Invert Eq. 35: beta from the relative curvature (Eq. 34) and tau0 from
    the peak position (Eq. 31). Returns (nan, nan) when the curvature is not
    negative."""
    if not curvature < 0.0:
        return math.nan, math.nan
    beta = math.sqrt(-curvature)
    return beta, math.exp(beta * (x_peak - 1.0))


# ------------------------------------------------------------------ smoothing
def lowpass_coefficients(s, k_c):
    """Real DFT of the binned spectrum (numpy's FFT), modes 0..k_c:
    a_k = sum_j s_j cos(2 pi j k / n), b_k = sum_j s_j sin(2 pi j k / n)."""
    s = np.asarray(s, dtype=np.float64)
    n = s.size
    if not 1 <= k_c < n / 2:
        raise ValueError("k_c must satisfy 1 <= k_c < n / 2")
    c = np.fft.rfft(s)[:k_c + 1]
    return c.real.copy(), -c.imag.copy()


def lowpass(s, k_c):
    """The low-passed spectrum on the bin centres: inverse real FFT of the
    spectrum's modes 0..k_c (higher modes set to zero)."""
    s = np.asarray(s, dtype=np.float64)
    c = np.fft.rfft(s)
    c[k_c + 1:] = 0.0
    return np.fft.irfft(c, n=s.size)


def smooth_derivatives(a, b, n, u):
    """Value and first two derivatives, in bin units, of the trigonometric
    polynomial s(u) = (1/n) [a_0 + 2 sum_{k>=1} (a_k cos(w_k u) + b_k sin(w_k u))],
    w_k = 2 pi k / n, at the fractional bin index u."""
    k = np.arange(a.size, dtype=np.float64)
    w = 2.0 * math.pi * k / n
    cw, sw = np.cos(w * u), np.sin(w * u)
    g = np.where(k == 0, 1.0, 2.0) / n
    s0 = np.sum(g * (a * cw + b * sw))
    s1 = np.sum(g * w * (-a * sw + b * cw))
    s2 = np.sum(g * w * w * (-a * cw - b * sw))
    return s0, s1, s2


def extract_peak(s, v_lo, v_hi, v_fs, k_c, x_min=None, x_max=None):
    """Main-peak extraction from one binned spectrum (n uniform bins over
    [v_lo, v_hi], bin centres v_j = v_lo + (j + 1/2) dv).

    Returns a dict: x_peak (v / v_fs), i_peak (smoothed value), curvature
    (I''/I in x), beta, tau0 (Eq. 35) and status."""
    s = np.asarray(s, dtype=np.float64)
    n = s.size
    dv = (v_hi - v_lo) / n
    a, b = lowpass_coefficients(s, k_c)
    sm = lowpass(s, k_c)
    xc = (v_lo + (np.arange(n) + 0.5) * dv) / v_fs
    lo = 0 if x_min is None else int(np.searchsorted(xc, x_min, side="left"))
    hi = n - 1 if x_max is None else int(np.searchsorted(xc, x_max, side="right")) - 1
    res = dict(x_peak=math.nan, i_peak=math.nan, curvature=math.nan, beta=math.nan,
               tau0=math.nan, status=STATUS_NO_PEAK, j_max=-1)
    if hi < lo:
        return res
    j = lo + int(np.argmax(sm[lo:hi + 1]))
    res["j_max"] = j
    if not sm[j] > 0.0:
        return res
    if j == lo or j == hi:
        res["status"] = STATUS_EDGE
        return res
    u = float(j)
    for _ in range(NEWTON_STEPS):
        _, d1, d2 = smooth_derivatives(a, b, n, u)
        if not d2 < 0.0:
            break
        u = min(max(u - d1 / d2, j - 1.0), j + 1.0)
    s0, _, s2 = smooth_derivatives(a, b, n, u)
    scale = (v_fs / dv) ** 2
    curv = s2 / s0 * scale
    res.update(x_peak=(v_lo + (u + 0.5) * dv) / v_fs, i_peak=s0, curvature=curv)
    if not curv < 0.0:
        res["status"] = STATUS_NOT_MAX
        return res
    res["beta"], res["tau0"] = params_from_peak(res["x_peak"], curv)
    res["status"] = STATUS_OK
    return res
