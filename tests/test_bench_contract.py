"""bench.py's reference arm (the FP64 oracle timed on the host cores, no
GPU): one JSON line with the contract's keys, the same metric, unit and
workload as the GPU line, a cpu_baseline describing the run and an e2e
object with zero host-device bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "scatter events/s"
    assert "cfg2" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_and_gpu_arms_share_the_config():
    """Both arms describe the workload with the same dict (workload_config)."""
    sys.path.insert(0, ROOT)
    import bench
    import argparse
    ns = argparse.Namespace(packets=1e8, snapshots=50)
    wl = bench.workload(ns)
    a, b = bench.workload_config(wl, 1), bench.workload_config(wl, 1)
    assert a == b and "l2" in a and a["snapshots"] == 50


def test_merged_bin_test_statistic():
    """The low-count two-sample test of the precision leg: identical
    histograms give chi^2 = 0; two Poisson samples of one spectrum give chi^2
    per group near 1 and no 5-sigma group; a 30 % excess in one region is
    found."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    rate = np.exp(-np.linspace(0, 6, 600)) * 40.0
    a = rng.poisson(rate).astype(float)
    b = rng.poisson(rate * 2).astype(float)              # twice the packets
    same = bench.merged_bin_test(a, 1e6, a, 1e6)
    assert same["chi2_per_group"] == 0.0 and same["max_abs_z"] == 0.0
    r = bench.merged_bin_test(a, 1e6, b, 2e6)
    assert 0.6 < r["chi2_per_group"] < 1.5 and r["pass_5sigma"], r
    assert r["groups"] > 50
    c = b.copy()
    c[:100] *= 1.3
    bad = bench.merged_bin_test(a, 1e6, rng.poisson(c).astype(float), 2e6)
    assert bad["chi2_per_group"] > 2.0 * r["chi2_per_group"], bad
    assert bad["max_abs_z"] > bad["bonferroni_z_1e-3"] > r["max_abs_z"], bad


def test_served_error_counts_moved_weight():
    """The serving line's check of served requests: tallies equal to the
    oracle's report no differing bin; a tally with one packet's weight moved
    by one bin (planted in the oracle's output) reports two bins and the moved
    share."""
    import math
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as O
    from paper_2012_00963_gb300 import workloads as W
    arr = [a for a in W.cfg5_arrivals(duration=1.0) if a.n_packets <= 150_000][:2]
    kept = []
    for k, a in enumerate(arr):
        wl = W.cfg5_request(a, r_ap=0.0, cone_alpha=math.pi / 2).replace(n_packets=20_000)
        kept.append((k, wl, np.pad(O.simulate(wl, spread_runs=0)["hist"], ((0, 0), (1, 1)))))
    ok = bench.served_error(kept, n_each=1)
    assert ok["bins_differing"] == 0 and ok["l1_rel"] == 0.0 and len(ok["requests"]) == 2
    k, wl, raw = kept[1]
    bad = raw.copy()
    j = int(np.argmax(bad[0]))
    bad[0, j] -= np.uint64(1 << 32)
    bad[0, j + 1] += np.uint64(1 << 32)
    r = bench.served_error([kept[0], (k, wl, bad)], n_each=1)
    tot = sum(float(x[2].sum()) for x in kept) / 2.0**32
    assert r["bins_differing"] == 2 and abs(r["l1_rel"] - 2.0 / tot) < 1e-12, r
