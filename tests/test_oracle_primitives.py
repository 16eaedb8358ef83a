"""Pins for the oracle's building blocks, each against something other than
the oracle itself: published known-answer vectors, textbook worked examples,
closed forms, independent quadrature and limiting cases."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from oracle import oracle as O
from paper_2012_00963_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with Random123
    (Salmon et al., SC'11): zero, all-ones and pi-digit counters/keys."""
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert list(O.philox4x32_10(ctr, key)) == want


def test_philox_uniformity():
    """Words from consecutive counters are uniform: chi-square over 256 cells
    of the top byte and a KS test of the 23-bit uniforms."""
    words = np.array([O.philox4x32_10([i, 0, 7, 3], [11, 13]) for i in range(20000)],
                     dtype=np.uint64).ravel()
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, 255)
    u = ((words >> 9).astype(np.float64) + 0.5) / 2.0**23
    assert stats.kstest(u, "uniform").pvalue > 1e-4


# ----------------------------------------------------------------- profiles
def _problem(**kw):
    return O.Problem(W.cfg1(**kw))


@pytest.mark.parametrize("beta,v_fs,v_max", [(5.0, 2000.0, 6000.0), (3.0, 2000.0, 0.0),
                                             (10.0, 1500.0, 0.0)])
def test_exponential_inverse_matches_quadrature(beta, v_fs, v_max):
    """v(s) from the oracle equals the root of the numerically integrated
    Eq. 20 mass fraction (scipy quad + brentq)."""
    pr = _problem(beta=beta, v_fs=v_fs, v_max=v_max)
    c = pr.constants()
    vb, vt = c["v_bot"], c["v_top"]
    if v_max == 0.0:
        # tail rule: the mass above v_top is 1e-6 of the untruncated law
        tail = integrate.quad(lambda v: beta / v_fs * np.exp(-beta * (v / v_fs - 1)), vt,
                              vt + 60 * v_fs / beta, epsabs=0, epsrel=1e-13, limit=200)[0]
        assert tail == pytest.approx(1e-6, rel=1e-9)
    f = lambda v: np.exp(-beta * (v / v_fs - 1.0))
    tot = integrate.quad(f, vb, vt, epsabs=0, epsrel=1e-13, limit=200)[0]
    for s in [1e-9, 1e-4, 0.01, 0.3, 0.5, 0.9, 0.999, 1 - 1e-7]:
        g = lambda v: integrate.quad(f, vb, v, epsabs=0, epsrel=1e-13, limit=200)[0] / tot - s
        v_ref = optimize.brentq(g, vb, vt, xtol=1e-10, rtol=1e-15)
        assert pr.inverse(s) == pytest.approx(v_ref, rel=1e-9, abs=1e-7)
        assert pr.cdf(v_ref) == pytest.approx(s, rel=1e-8, abs=1e-12)


def test_tabulated_inverse_matches_quadrature():
    """Piecewise-linear dm/dv: the exact quadratic inversion agrees with
    quad + brentq on np.interp of the same points."""
    pv = np.array([2100.0, 2500.0, 3000.0, 3200.0, 5000.0])
    pf = np.array([3.0, 1.0, 2.5, 0.2, 0.05])
    pr = _problem(profile_kind="tabulated", prof_v=pv, prof_f=pf, v_max=0.0)
    c = pr.constants()
    assert c["v_bot"] == 2100.0 and c["v_top"] == 5000.0
    f = lambda v: np.interp(v, pv, pf)
    tot = integrate.quad(f, pv[0], pv[-1], points=pv[1:-1], epsrel=1e-13)[0]
    for s in [1e-6, 0.1, 0.37, 0.6, 0.95, 0.99999]:
        g = lambda v: integrate.quad(f, pv[0], v, points=[p for p in pv[1:-1] if p < v],
                                     epsrel=1e-13)[0] / tot - s
        v_ref = optimize.brentq(g, pv[0], pv[-1], xtol=1e-10)
        assert pr.inverse(s) == pytest.approx(v_ref, rel=1e-9)


def test_optical_depth_from_particle_sums():
    """Eq. 8-10 with explicit sums over a sampled log-normal population
    converge to the oracle's closed-form optical depth 3 m0 Q / (2 rho d_s)."""
    rng = np.random.default_rng(0)
    for d_m, sig in [(2e-6, 0.0), (3e-6, 0.5), (1.5e-6, 0.3)]:
        pr = _problem(d_m=d_m, sigma_ln=sig, m0=5 * W.MG_CM2)
        c = pr.constants()
        d = d_m * np.exp(sig * rng.standard_normal(4_000_000))
        m0, rho, q = 5 * W.MG_CM2, 7290.0, 2.0
        tau_sum = 3 * m0 * np.sum(d**2 * q) / (2 * rho * np.sum(d**3))
        assert c["tau_tot"] == pytest.approx(tau_sum, rel=3e-3 if sig else 1e-12)
    # the benchmark cloud: 0.5 mg/cm^2 of 2 um tin spheres with Q_ext = 2
    assert _problem().constants()["tau_tot"] == pytest.approx(1.0288065843621399, rel=1e-14)


# ----------------------------------------------------------------- Mie
def test_mie_textbook_example():
    g = json.load(open(os.path.join(GOLDEN, "mie_bohren_huffman.json")))
    x = 2 * np.pi * g["radius_um"] / g["wavelength_um"]
    q, *_ = O.mie_single(x, complex(g["m_re"], g["m_im"]))
    assert q[0] == pytest.approx(g["q_ext"], rel=g["rtol"])
    assert q[1] == pytest.approx(g["q_sca"], rel=g["rtol"])
    assert q[2] == pytest.approx(g["q_back"], rel=g["rtol"])


@pytest.mark.parametrize("m", [1.5 + 0.01j, 3.0 + 9.0j, 1.33 + 0.0j])
def test_mie_rayleigh_limit(m):
    """x -> 0: Q_sca = 8/3 x^4 |K|^2 and Q_abs = 4 x Im K, K = (m^2-1)/(m^2+2)."""
    x = 1e-3
    q, *_ = O.mie_single(x, m)
    K = (m * m - 1) / (m * m + 2)
    assert q[1] == pytest.approx(8 / 3 * x**4 * abs(K) ** 2, rel=1e-4)
    if m.imag > 0:
        assert q[0] - q[1] == pytest.approx(4 * x * K.imag, rel=1e-3)


@pytest.mark.parametrize("x,m", [(0.5, 1.5 + 0.1j), (5.0, 3.0 + 9.0j), (30.0, 3.0 + 9.0j),
                                 (12.0, 1.33 + 0.0j)])
def test_mie_angular_consistency(x, m):
    """Angular functions against the coefficient sums: Q_sca = (1/x^2) int
    (|S1|^2+|S2|^2) sin, g from the same integral, optical theorem through
    S1(0) = S2(0), backscatter through S1(pi); Q_abs >= 0; real m conserves."""
    th = np.linspace(0, np.pi, 20001)
    mu = np.cos(th)
    q, s11, s22, s0, n = O.mie_single(x, m, mu)
    w = (s11 + s22) * np.sin(th)
    qsca_int = integrate.simpson(w, x=th) / x**2
    g_int = integrate.simpson(w * mu, x=th) / (x**2 * q[1])
    assert qsca_int == pytest.approx(q[1], rel=1e-6)
    assert g_int == pytest.approx(q[3], rel=1e-5, abs=1e-7)
    assert s11[0] == pytest.approx(s22[0], rel=1e-12)
    assert s11[0] == pytest.approx(abs(s0) ** 2, rel=1e-10)
    assert q[0] == pytest.approx(4 / x**2 * s0.real, rel=1e-12)
    assert q[2] == pytest.approx(4 * s11[-1] / x**2, rel=1e-9)
    assert q[0] - q[1] >= -1e-12
    if m.imag == 0:
        assert q[0] == pytest.approx(q[1], rel=1e-10)


def test_mie_large_sphere_extinction():
    """Extinction paradox: Q_ext -> 2 for x >> 1, approached through the edge
    term that decays like x^(-2/3) (van de Hulst)."""
    for x in [1000.0, 8000.0]:
        q, *_ = O.mie_single(x, 3.0 + 9.0j)
        assert 2.0 < q[0] < 2.0 + 5.0 * x ** (-2.0 / 3.0)
        assert (q[0] - 2.0) * x ** (2.0 / 3.0) > 2.0


def test_mie_table_size_average():
    """The size-averaged table: 2 pi int p sin = <C_sca> (its normalisation);
    q_ext and albedo equal an independent scipy quadrature over the number
    log-normal of d^2 Q(d); sigma = 0 reduces to the single sphere."""
    lam, d_m, sig, m = 1550e-9, 3e-6, 0.5, 3 + 9j
    th, p, qext, alb, g = O.mie_table(m, lam, d_m, sig, n_angle=1801, n_size=256)
    lo, hi = np.log(d_m) - 6 * sig, np.log(d_m) + 6 * sig
    pdf = lambda y: np.exp(-0.5 * ((y - np.log(d_m)) / sig) ** 2) / (np.sqrt(2 * np.pi) * sig)

    def qq(y):
        return O.mie_single(np.pi * np.exp(y) / lam, m)[0]

    ys = np.linspace(lo, hi, 1201)
    Q = np.array([qq(y) for y in ys])
    d2 = np.exp(2 * ys) * pdf(ys)
    A2 = integrate.simpson(d2, x=ys)
    Aext = integrate.simpson(d2 * Q[:, 0], x=ys)
    Asca = integrate.simpson(d2 * Q[:, 1], x=ys)
    assert qext == pytest.approx(Aext / A2, rel=1e-7)
    assert alb == pytest.approx(Asca / Aext, rel=1e-7)
    csca = np.pi / 4 * Asca
    assert 2 * np.pi * integrate.simpson(p * np.sin(th), x=th) == pytest.approx(csca, rel=1e-4)
    # monodisperse
    th1, p1, qext1, alb1, g1 = O.mie_table(m, lam, 1e-6, 0.0, n_angle=181)
    q1, *_ = O.mie_single(np.pi * 1e-6 / lam, m)
    assert qext1 == pytest.approx(q1[0], rel=1e-14)
    assert alb1 == pytest.approx(q1[1] / q1[0], rel=1e-14)
    assert g1 == pytest.approx(q1[3], rel=1e-14)


# ----------------------------------------------------------------- phase sampling
def test_hg_table_normalised():
    th, p = O.hg_table(0.7, 1801)
    assert 2 * np.pi * integrate.simpson(p * np.sin(th), x=th) == pytest.approx(1.0, rel=1e-6)


def test_phase_sampler_hg_closed_form():
    """Samples of cos(theta) from the integer inverse CDF follow the closed-form
    Henyey–Greenstein CDF (KS), their mean is g_tab (4 sigma), and g_tab is
    the HG asymmetry 0.7 up to the table's O(dtheta^2)."""
    g = 0.7
    th, p = O.hg_table(g, 1801)
    cq, g_tab = O.phase_cdf(th, p)
    assert cq[0] == 0 and cq[-1] == 2**24 and np.all(np.diff(cq.astype(np.int64)) >= 0)
    assert g_tab == pytest.approx(g, abs=2e-5)
    rng = np.random.default_rng(1)
    ms = rng.integers(0, 2**24, 40000)
    c = np.cos([O.phase_sample(th, cq, int(m)) for m in ms])
    hg_cdf = lambda mu: (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    assert stats.kstest(c, hg_cdf).pvalue > 1e-4
    assert abs(c.mean() - g_tab) < 4 * c.std() / np.sqrt(len(c))


def test_phase_sampler_bin_edges():
    """m at a CDF step lands at the start of its bin; the last m stays inside;
    cells of zero probability are never sampled."""
    th = np.linspace(0, np.pi, 5)
    p = np.array([1.0, 1.0, 0.0, 0.0, 1.0])
    cq, _ = O.phase_cdf(th, p)
    assert cq[2] == cq[3] == cq[4] == 2**24       # cells 2 and 3 carry no weight
    assert O.phase_sample(th, cq, int(cq[1])) == pytest.approx(
        th[1] + 0.5 / (int(cq[2]) - int(cq[1])) * (th[2] - th[1]), rel=1e-15)
    for m in [0, int(cq[1]) - 1, int(cq[1]), 2**24 - 1]:
        t = O.phase_sample(th, cq, m)
        assert th[0] < t < th[2]
    t = np.array([O.phase_sample(th, cq, m) for m in range(0, 2**24, 4099)])
    assert np.all(t < th[2])


# ----------------------------------------------------------------- rotation
def test_rotation_geometry():
    rng = np.random.default_rng(2)
    for _ in range(200):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        th = rng.uniform(0, np.pi)
        ph = rng.uniform(0, 2 * np.pi)
        v = O.rotate(u, np.cos(th), np.sin(th), np.cos(ph), np.sin(ph))
        assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-14)
        assert np.dot(u, v) == pytest.approx(np.cos(th), abs=1e-12)
    # azimuthal average of the new direction is cos(theta) u
    u = np.array([0.3, -0.5, 0.6])
    u /= np.linalg.norm(u)
    th = 1.1
    phis = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
    vs = np.array([O.rotate(u, np.cos(th), np.sin(th), np.cos(f), np.sin(f)) for f in phis])
    assert np.allclose(vs.mean(axis=0), np.cos(th) * u, atol=1e-12)
    # Eq. 17 branch for a vertical packet keeps the sign of u_z
    v = O.rotate([0, 0, -1.0], np.cos(0.3), np.sin(0.3), 1.0, 0.0)
    assert v[2] == pytest.approx(-np.cos(0.3)) and v[0] == pytest.approx(np.sin(0.3))


@pytest.mark.parametrize("eps", [1e-3, 1.4e-3, 1e-6, 1e-9, 1e-13])
def test_rotation_is_continuous_at_the_pole(eps):
    """Near the pole the rotation keeps the exact scattering angle, and the
    new direction tends to the vertical packet's as the tilt goes to zero, with
    the azimuth measured from the tilt's own direction alpha (the limit of the
    Eq. 16 frame): no jump at any tilt (the tilt eps = 1.4e-3 is the old
    switch to Eq. 17 at 1 - |u_z| = 1e-6)."""
    alpha, th, ph = 0.7, 0.9, 2.1
    u = np.array([eps * np.cos(alpha), eps * np.sin(alpha), -np.sqrt(1.0 - eps * eps)])
    v = O.rotate(u, np.cos(th), np.sin(th), np.cos(ph), np.sin(ph))
    assert np.dot(u, v) == pytest.approx(np.cos(th), abs=1e-12)
    e1 = np.array([-np.cos(alpha), -np.sin(alpha), 0.0])   # limit of (u_x u_z, u_y u_z, -s^2) / s
    e2 = np.array([-np.sin(alpha), np.cos(alpha), 0.0])
    lim = np.sin(th) * (np.cos(ph) * e1 + np.sin(ph) * e2) + np.cos(th) * np.array([0, 0, -1.0])
    assert np.allclose(v, lim, atol=3.0 * eps + 1e-12)
