"""Spectrograms: the PDV spectrum over many snapshot times (the v-t image of
the paper's Fig. 1 and Fig. 16(a)).

The cloud is self-similar (z = v t), so the library transports every packet
once and tests it at all snapshot times; a spectrogram is one
``pdv_simulate_spectrum`` call with up to 4096 snapshot times, its rows the
spectra at those times. This module only marshals that call and writes the
image (binary PGM, or the raw array with numpy).
"""
from __future__ import annotations

import numpy as np

from . import pdv


def spectrogram(ctx: "pdv.Context", cloud: "pdv.Cloud", wl, t_snap, per_dv: bool = False,
                precision=None) -> dict:
    """Run one request over the snapshot times ``t_snap`` (seconds). Returns
    ``image`` [n_t, n_bins] (the normalised spectra, rows in the order of
    ``t_snap``), ``raw`` tallies and ``counters``, plus the axes."""
    t = np.asarray(t_snap, dtype=np.float64)
    r = pdv.simulate_spectrum(ctx, cloud, wl, snapshots=t, per_dv=per_dv, precision=precision)
    dv = (wl.v_hi - wl.v_lo) / wl.n_bins
    return {"image": r["spectrum"], "raw": r["raw"], "counters": r["counters"], "t": t,
            "v": wl.v_lo + (np.arange(wl.n_bins) + 0.5) * dv}


def to_gray(image, log_range: float = 4.0) -> np.ndarray:
    """8-bit gray levels of an image: log10 scale over ``log_range`` decades
    below the maximum (0 below that, 255 at the maximum); linear when
    ``log_range`` is 0. An all-zero image maps to 0."""
    a = np.asarray(image, dtype=np.float64)
    top = float(a.max()) if a.size else 0.0
    if not top > 0.0:
        return np.zeros(a.shape, dtype=np.uint8)
    if log_range > 0.0:
        with np.errstate(divide="ignore"):
            x = (np.log10(np.maximum(a, 0.0) / top) + log_range) / log_range
    else:
        x = np.maximum(a, 0.0) / top
    return np.clip(np.rint(255.0 * x), 0, 255).astype(np.uint8)


def write_pgm(path: str, image, log_range: float = 4.0, time_up: bool = True) -> None:
    """Write an image as a binary PGM (P5): columns are velocity bins, rows
    are snapshot times (the latest at the top when ``time_up``)."""
    g = to_gray(image, log_range)
    if g.ndim != 2:
        raise ValueError("a spectrogram is two-dimensional")
    if time_up:
        g = g[::-1]
    h, w = g.shape
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (w, h))
        f.write(np.ascontiguousarray(g).tobytes())


def read_pgm(path: str) -> np.ndarray:
    """Read back a binary PGM written by ``write_pgm``."""
    with open(path, "rb") as f:
        data = f.read()
    parts = data.split(b"\n", 3)
    if parts[0] != b"P5":
        raise ValueError("not a binary PGM")
    w, h = (int(x) for x in parts[1].split())
    if int(parts[2]) != 255:
        raise ValueError("only 8-bit PGM is supported")
    return np.frombuffer(parts[3][: w * h], dtype=np.uint8).reshape(h, w)
