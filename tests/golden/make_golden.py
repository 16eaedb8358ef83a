"""Write the oracle-generated reference spectra stored under tests/golden/.

Calls only the FP64 oracle (oracle/). Run from the repository root:

    python tests/golden/make_golden.py [serving] [precision]

* serving_target.npz — the synthetic "measured" spectrum that the serving
  benchmark fits: the served request shape (HG g = 0.7, albedo 0.6,
  Q_ext = 2, 400 bins over 0-8000 m/s, t = 1 us, every upward photon
  counted as the paper does) with the hidden parameters beta = 6,
  m0 = 3 mg/cm^2, d = 2 um, 1e7 packets (seed 77).
* precision_cfg3.npz — the heavy multiple-scattering cloud (20 mg/cm^2 of
  1 um tin, beta = 3, Mie m = 3 + 9i) at 1e7 packets: the reference for the
  per-bin error of the GPU paths. It draws seed 303, so its packets are
  independent of the GPU runs' (seed 3) and the comparison is between two
  independent Monte Carlo samples.
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2012_00963_gb300 import workloads as W  # noqa: E402

SERVING_HIDDEN = dict(beta=6.0, m0=3.0 * W.MG_CM2, d_m=2.0 * W.UM)
SERVING_PROBE = dict(r_ap=0.0, cone_alpha=math.pi / 2)     # every upward photon (Eq. 19)


def serving_workload(beta, m0, d_m, n_packets, seed):
    a = W.Arrival(t=0.0, beta=beta, m0=m0, d_m=d_m, n_packets=n_packets, seed=seed)
    return W.cfg5_request(a, **SERVING_PROBE)


PRECISION_SEED = 303


def precision_workload(n_packets, seed=PRECISION_SEED):
    return W.cfg3(n_packets=n_packets, r_ap=3.0 * W.MM, cone_alpha=0.5, seed=seed)


def save(name, wl, res, seconds):
    np.savez_compressed(
        os.path.join(HERE, name), hist=res["hist"], counters=res["counters"],
        n_packets=wl.n_packets, v_lo=wl.v_lo, v_hi=wl.v_hi, n_bins=wl.n_bins,
        tau_tot=res["tau_tot"], seconds=seconds, seed=wl.seed,
        note="FP64 oracle (oracle/pdv_oracle.c) written by tests/golden/make_golden.py")


def main(which):
    if "serving" in which:
        wl = serving_workload(n_packets=10_000_000, seed=77, **SERVING_HIDDEN)
        t = time.time()
        res = O.simulate(wl)
        save("serving_target.npz", wl, res, time.time() - t)
        print("serving target", time.time() - t, "s", res["counters"][0][:6])
    if "precision" in which:
        wl = precision_workload(10_000_000)
        t = time.time()
        res = O.simulate(wl, table=O.phase_table(wl))
        save("precision_cfg3.npz", wl, res, time.time() - t)
        print("precision cfg3", time.time() - t, "s", res["counters"][0][:6])


if __name__ == "__main__":
    main(sys.argv[1:] or ["serving", "precision"])
