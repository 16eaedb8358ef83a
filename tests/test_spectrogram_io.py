"""The spectrogram image writer (host-side formatting only)."""
import numpy as np

from paper_2012_00963_gb300 import spectrogram as S


def test_gray_levels():
    img = np.array([[1.0, 1e-2, 1e-4, 1e-6], [0.0, 0.5, 1e-3, -1.0]])
    g = S.to_gray(img, log_range=4.0)
    assert g[0, 0] == 255 and g[0, 2] == 0 and g[0, 3] == 0 and g[1, 0] == 0 and g[1, 3] == 0
    assert g[0, 1] == 128                      # two of four decades below the top
    lin = S.to_gray(img, log_range=0.0)
    assert lin[1, 1] == 128 and lin[0, 0] == 255
    assert not S.to_gray(np.zeros((3, 4))).any()


def test_pgm_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    img = rng.random((7, 11))
    p = tmp_path / "s.pgm"
    S.write_pgm(str(p), img, log_range=2.0)
    head = open(p, "rb").read(12)
    assert head.startswith(b"P5\n11 7\n255\n")
    back = S.read_pgm(str(p))
    assert np.array_equal(back, S.to_gray(img, 2.0)[::-1])   # latest time at the top
    S.write_pgm(str(p), img, log_range=2.0, time_up=False)
    assert np.array_equal(S.read_pgm(str(p)), S.to_gray(img, 2.0))
