"""Error bound of the transport kernel's own sin(pi y), cos(pi y) for y in
[0, 2] (sincospi_half_turns in pdv_internal.cuh): its binary32 operation
sequence is replayed here with the coefficients read from the header (each
fused multiply-add formed exactly in binary64 and rounded once to binary32),
and compared with the FP64 library values on a dense grid and at the
quarter turns."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2012_00963_gb300", "csrc", "pdv_internal.cuh")
F32 = np.float32


def _coefficients():
    src = open(HDR).read()
    body = src[src.index("void sincospi_half_turns"):]
    body = body[:body.index("\n}\n")]
    lits = [float(x) for x in re.findall(r"(-?\d+\.\d+)f", body)]
    # rint(2 y), fmaf(-0.5, q, y), then the sine and cosine polynomials
    assert lits[:2] == [2.0, -0.5], lits[:2]
    return np.array(lits[2:6], F32), np.array(lits[6:10], F32), lits[10]


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def _sincospi(y):
    ps_c, pc_c, one = _coefficients()
    assert one == 1.0
    y = y.astype(F32)
    q = np.rint(F32(2.0) * y).astype(F32)
    r = _fma(F32(-0.5), q, y)
    t = (r * r).astype(F32)
    p = _fma(t, ps_c[0], ps_c[1])
    p = _fma(t, p, ps_c[2])
    p = _fma(t, p, ps_c[3])
    sr = (p * r).astype(F32)
    h = _fma(t, pc_c[0], pc_c[1])
    h = _fma(t, h, pc_c[2])
    h = _fma(t, h, pc_c[3])
    cr = _fma(t, h, F32(1.0))
    iq = q.astype(np.int64) & 3
    a = np.where(iq & 1, cr, sr)
    b = np.where(iq & 1, sr, cr)
    return np.where(iq & 2, -a, a), np.where((iq + 1) & 2, -b, b)


def test_error_bound_on_a_dense_grid():
    rng = np.random.default_rng(7)
    y = np.concatenate([rng.random(2_000_000).astype(F32) * 2,
                        np.linspace(0.0, 2.0, 1_000_001).astype(F32)])
    s, c = _sincospi(y)
    yd = y.astype(np.float64)
    es = np.abs(s - np.sin(np.pi * yd))
    ec = np.abs(c - np.cos(np.pi * yd))
    assert es.max() <= 1.0e-7 and ec.max() <= 1.0e-7, (es.max(), ec.max())
    assert np.all(np.abs(s) <= 1.0) and np.all(np.abs(c) <= 1.0)


def test_quarter_turns_are_exact():
    y = np.array([0.0, 0.5, 1.0, 1.5, 2.0], F32)
    s, c = _sincospi(y)
    assert np.array_equal(np.abs(s), [0.0, 1.0, 0.0, 1.0, 0.0])
    assert np.array_equal(c, [1.0, 0.0, -1.0, 0.0, 1.0]) or np.array_equal(np.abs(c), [1.0, 0.0, 1.0, 0.0, 1.0])
    assert np.array_equal(np.sign(s[[1, 3]]), [1.0, -1.0]) and np.array_equal(c[[0, 2, 4]], [1.0, -1.0, 1.0])
