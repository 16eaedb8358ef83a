#!/usr/bin/env python
"""Benchmark of the PDV Monte Carlo hot path on GB300.

Workload (default): the log-normal Mie cloud of the benchmark set — d_m = 3 um,
sigma = 0.5, m = 3 + 9i at 1550 nm, 5 mg/cm^2 of tin, beta = 5 (mass tail
1e-6), 50 snapshots at 0.5-5 us, 1e8 packets per snapshot, 600 bins over
0-8000 m/s, FP32 transport.

One step = one pass of every step of the path: the cloud's mass table (FP64
kernel), the phase CDF (FP64 kernel), the persistent FP32 transport of all
packets with detection at all 50 snapshot times, and the normalisation to 50
spectra. ``value`` is measured with device-resident inputs and device outputs;
``e2e`` runs the same step through the public API with pinned host inputs and
host outputs (copies inside the timed region).

Unit: scatter events per second, counted once per packet history (a history
serves every snapshot time). Also reported: all events/s, spectra/s, the
plain FP64 GPU path on the same workload, the issue-rate roofline of the
transport kernel, and the FP64 CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon scatter events/s & spectra/s vs plain FP64 path; p50/p99 request latency"
UNIT = "scatter events/s"
# Algorithmic thread-instructions of one event (a flight and what ends it) on
# the FP32 path, each operation of the method counted once: Philox4x32-10 with
# its counter set-up (64), the free path's uniform, logarithm, fixed-point
# step and escape/surface test (20), the velocity inversion (12), the lateral
# move (5), the albedo test (2), the phase-table inversion and theta (16),
# sin/cos of theta and phi (30), the rotation and renormalisation (25), the
# compensated Doppler sum (8) and the event bookkeeping (18): 200, the top of
# the 150-200 range of the analysis.
ALGO_INST_PER_EVENT = 200.0
SCHEDULERS, LANES, F_NOMINAL_MHZ = 4, 32, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=float, default=1e8, help="packets per snapshot")
    ap.add_argument("--snapshots", type=int, default=50)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mode", default="default",
                    choices=["default", "serve", "batch", "precision", "model", "extract-mc",
                             "stepping", "spectrogram", "cpu-baseline", "fig12", "fig6", "trends",
                             "implicit"])
    ap.add_argument("--times", type=int, default=512, help="snapshot times of the spectrogram mode")
    ap.add_argument("--out", default="", help="spectrogram mode: write the v-t image (PGM) here")
    ap.add_argument("--model-sets", type=int, default=100_000,
                    help="parameter sets / spectra of the model mode")
    ap.add_argument("--extract-simt", action="store_true",
                    help="model mode: the extraction's products on the CUDA cores")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sets", type=int, default=256)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-side-legs", dest="side_legs", action="store_false",
                    help="default mode: skip the short precision and batch legs")
    return ap.parse_args()


def workload(args, rank=0):
    import numpy as np
    from paper_2012_00963_gb300 import workloads as W
    t = tuple(np.linspace(0.5, 5.0, args.snapshots) * W.US)
    return W.cfg2(n_packets=int(args.packets), t_snap=t, seed=2 + 1000 * rank)


def reduce_max(values, world):
    """Element-wise maximum over ranks of a float64 tensor (the slowest rank's
    times set the whole job's rate); identity on one process."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(values, op=dist.ReduceOp.MAX)
    return values


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def source_hash():
    h = hashlib.sha1()
    for f in ("transport.cu", "pdv_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2012_00963_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profile_counters():
    """Per-event DRAM traffic and issued instructions of the transport kernel
    from the committed ncu summary, if it was taken on the current source."""
    p = os.path.join(ROOT, "profiles", "transport_f32_counters.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d if d.get("source_hash") == source_hash() else None


# ----------------------------------------------------------------------- CPU
def oracle_sample(wl, seconds, threads):
    """Time the FP64 oracle on a bounded sample of the workload (all snapshot
    times, a slice of the packets), sized for about `seconds` of wall time."""
    from oracle import oracle as O
    table = O.phase_table(wl)
    n = 200
    while True:
        t0 = time.perf_counter()
        r = O.simulate(wl, n_threads=threads, n_packets=n, table=table)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.5 or n >= wl.n_packets:
            break
        n = min(int(n * max(2.0, 0.8 * seconds / max(dt, 1e-3))), wl.n_packets)
    ns = len(wl.t_snap)
    scat = int(r["counters"][0][2])          # scatters of the n distinct histories
    return dict(value=scat / dt, packets=n, seconds=dt, snapshots=ns,
                spectra_per_s=ns * (n / wl.n_packets) / dt,
                events_per_s=int(r["counters"][0][1]) / dt, result=r)


def workload_config(wl, world):
    """The benchmark workload as both arms report it."""
    return {"workload": "cfg2: log-normal Mie cloud d_m=3um sigma=0.5 m=3+9i lambda=1550nm, "
                        "5 mg/cm^2 tin, beta=5, %d snapshots 0.5-5us, %.0e packets per snapshot, "
                        "%d bins 0-8000 m/s" % (len(wl.t_snap), wl.n_packets, wl.n_bins),
            "packets_per_snapshot": wl.n_packets, "snapshots": len(wl.t_snap), "bins": wl.n_bins,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "GPU arm: flushed between steps (256 MiB write)"}


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload(args)
    threads = os.cpu_count() or 1
    per_step = max(1.0, min(6.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(wl, per_step * 0.25, threads)
    vals, sp, tot, pk = [], [], 0.0, 0
    for _ in range(args.steps):
        s = oracle_sample(wl, per_step, threads)
        vals.append(s["value"])
        sp.append(s["spectra_per_s"])
        tot += s["seconds"]
        pk = s["packets"]
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(wl, world),
        "spectra_per_s": statistics.median(sp),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d packets x %d snapshots per step (of %d packets)" % (
                             pk, len(wl.t_snap), wl.n_packets)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------- GPU
def our_arm(args):
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = workload(args, rank)
    ns, nb = len(wl.t_snap), wl.n_bins
    NC = len(pdv.COUNTER_NAMES)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    ctx = pdv.Context(local, stream=stream.cuda_stream)
    # prerequisite input: the size-averaged Mie table (FP64 GPU kernel, once)
    table = pdv.phase_table(ctx, wl)
    th_pin = torch.from_numpy(np.ascontiguousarray(table[0])).pin_memory()
    p_pin = torch.from_numpy(np.ascontiguousarray(table[1])).pin_memory()
    dev_out = {"spectrum": torch.zeros(ns * nb, dtype=torch.float64, device=dev),
               "counters": torch.zeros(ns * NC, dtype=torch.int64, device=dev)}
    host_spec = torch.zeros(ns * nb, dtype=torch.float64).pin_memory()
    host_cnt = torch.zeros(ns * NC, dtype=torch.int64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    tbl = (th_pin.numpy(), p_pin.numpy(), table[2], table[3])

    def step(precision, device_outputs):
        cloud = pdv.Cloud(ctx, wl, table=tbl)            # a1-a3 on the device
        if device_outputs:
            req = pdv.Request(cloud, wl, precision=precision, device_out=dev_out)
        else:
            req = pdv.Request(cloud, wl, precision=precision, raw=False, counters=True)
            req.spectrum = host_spec.numpy().reshape(ns, nb)
            req.c.out_spectrum = host_spec.data_ptr()
        pdv.pdv_simulate_spectrum(ctx.handle, req.c)    # a4-a14
        ev = ctx.stats()["last_events"]
        cloud.close()
        return ev, ctx.stats()["last_transport_ms"]

    def scat_per_step():
        return int(dev_out["counters"].view(ns, NC)[0, 2].item())

    def timed(precision, device_outputs, steps, warmup):
        for _ in range(warmup):
            step(precision, device_outputs)
        barrier()
        l0 = ctx.stats()["kernel_launches"]
        times, kern, events = [], [], 0
        for _ in range(steps):
            flush.zero_()                                  # L2 flushed between steps
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ev, kms = step(precision, device_outputs)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            kern.append(kms)
            events += ev
        barrier()
        launches = ctx.stats()["kernel_launches"] - l0
        return times, kern, events, launches

    clocks = Clocks(local)
    # ---- device-resident value
    clocks.start()
    t_ms, k_ms, events, launches = timed("fp32", True, args.steps, args.warmup)
    clk = clocks.stop()
    scat = scat_per_step()
    total_s = sum(t_ms) / 1e3
    # ---- end to end through the public API with host buffers
    e_ms, _, _, _ = timed("fp32", False, max(2, args.steps // 2), 1)
    # ---- plain FP64 GPU path on the same workload
    f_ms, fk_ms, f_events, _ = timed("fp64", True, args.fp64_steps, 1)
    f_scat = scat_per_step()

    vals = torch.tensor([total_s, sum(e_ms) / 1e3, sum(f_ms) / 1e3], dtype=torch.float64,
                        device=dev)
    total_s, e_s, f_s = [float(x) for x in reduce_max(vals, world).cpu()]
    steps = args.steps
    value = world * scat * steps / total_s
    spectra = world * ns * steps / total_s
    e_steps = max(2, args.steps // 2)
    e2e_value = world * scat * e_steps / e_s
    f_value = world * f_scat * args.fp64_steps / f_s

    kern_ms = statistics.mean(k_ms)
    ev_per_launch = events / steps
    achieved = ALGO_INST_PER_EVENT * ev_per_launch / (kern_ms / 1e3) / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_mhz = (clk or {}).get("sm_max_mhz") or F_NOMINAL_MHZ
    peak = sms * SCHEDULERS * LANES * f_mhz * 1e6 / 1e9
    prof = profile_counters()
    traffic = prof["dram_bytes_per_event"] * ev_per_launch if prof else None
    issue_meas = pdv.pdv_measure_issue_rate(ctx.handle, 0.2) / 1e9   # after the timed region

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded cloud of the paper's workload shape; no dataset)",
        "config": workload_config(wl, world),
        "spectra_per_s": spectra,
        "events_per_s": world * (events / steps) * steps / total_s,
        "packet_histories_per_s": world * wl.n_packets * steps / total_s,
        "fp64_plain": {"value": f_value, "unit": UNIT, "ms_per_step": 1e3 * f_s / args.fp64_steps,
                       "spectra_per_s": world * ns * args.fp64_steps / f_s,
                       "kernel_ms": statistics.mean(fk_ms)},
        "speedup_vs_fp64_plain": value / f_value if f_value else None,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(th_pin.numel() * 8 + p_pin.numel() * 8 + ns * 8),
                "d2h_bytes_per_step": int(ns * nb * 8 + ns * 112)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Ginst/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_transport_f32", "kernel_ms": kern_ms,
                     "algo_inst_per_event": ALGO_INST_PER_EVENT,
                     "peak_basis": "%d SM (device) x %d schedulers x %d lanes x %.0f MHz (max SM "
                                   "clock sampled during the run): issue rate" % (
                                       sms, SCHEDULERS, LANES, f_mhz),
                     "peak_measured": issue_meas, "frac_of_measured": achieved / issue_meas,
                     "peak_measured_basis": "independent FP32 FMA chains, 64 warps per SM "
                                            "(pdv_measure_issue_rate)"},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        line["serving"] = serving_run(ctx, args.serve_seconds, args.rate)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(wl, args.cpu_seconds, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": os.cpu_count() or 1,
                                "kind": "oracle",
                                "sample": "%d packets x %d snapshots (%.1f s)" % (
                                    cb["packets"], cb["snapshots"], cb["seconds"]),
                                "spectra_per_s": cb["spectra_per_s"]}
        line["spectrum_error"] = same_packets_error(ctx, wl, tbl, cb)
    if rank == 0 and world == 1 and args.side_legs:
        line["precision"] = precision_leg(ctx, stream, 10_000_000)
        line["batch"] = batch_leg(ctx, stream, scale=0.1)
        line["model"] = model_leg(ctx, stream)
        line["stepping"] = stepping_leg(ctx, stream)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0



# ----------------------------------------------------------------------- error legs
def merged_bin_test(h_a, n_a, h_b, n_b, min_count=20.0):
    """Two-sample comparison of weight histograms (packet units) from n_a and
    n_b packets that is valid at low counts: adjacent bins are merged, left to
    right, until both samples hold at least `min_count` in the group (a short
    last group joins the one before). Per group z = (a/n_a - b/n_b) / sigma
    with the pooled rate; weights are at most one packet, so the Poisson
    variance used here bounds the true one from above. Returns chi^2 per group,
    the largest |z|, the groups, the Bonferroni bound for a 1e-3 family-wise
    false alarm over the groups, and whether max |z| stays below 5."""
    import numpy as np
    from statistics import NormalDist
    h_a = np.asarray(h_a, np.float64).ravel()
    h_b = np.asarray(h_b, np.float64).ravel()
    groups, ga, gb = [], 0.0, 0.0
    for x, y in zip(h_a, h_b):
        ga += x
        gb += y
        if ga >= min_count and gb >= min_count:
            groups.append([ga, gb])
            ga = gb = 0.0
    if groups and (ga or gb):
        groups[-1][0] += ga
        groups[-1][1] += gb
    if not groups:
        return {"groups": 0}
    g = np.asarray(groups)
    pooled = (g[:, 0] + g[:, 1]) / (n_a + n_b)
    z = (g[:, 0] / n_a - g[:, 1] / n_b) / np.sqrt(pooled * (1.0 / n_a + 1.0 / n_b))
    bonf = NormalDist().inv_cdf(1.0 - 1e-3 / (2.0 * len(g)))
    return {"groups": int(len(g)), "chi2_per_group": float(np.mean(z * z)),
            "max_abs_z": float(np.abs(z).max()), "bonferroni_z_1e-3": float(bonf),
            "pass_5sigma": bool(np.abs(z).max() < 5.0)}


def same_packets_error(ctx, wl, tbl, cb):
    """Spectrum error of the FP32 and the plain FP64 GPU paths against the FP64
    oracle on the oracle's own sample (the same packets, the same random
    numbers): the share of tallied weight that lands in a different bin or
    snapshot, per-bin z, and the bins that differ at all."""
    import numpy as np
    from paper_2012_00963_gb300 import pdv
    ref = cb["result"]
    n = cb["packets"]
    h_o = ref["hist"].astype(np.float64) / 2.0**32
    cloud = pdv.Cloud(ctx, wl, table=tbl)
    out = {"packets": n, "snapshots": len(wl.t_snap), "bins": wl.n_bins,
           "note": "the GPU paths and the oracle transport the same packets with the same "
                   "random numbers; differences come from rounding alone"}
    for prec in ("fp32", "fp64"):
        r = pdv.simulate_spectrum(ctx, cloud, wl, precision=prec, n_packets=n)
        h_g = r["raw"][:, 1:-1].astype(np.float64) / 2.0**32
        z = np.abs(h_g - h_o) / np.sqrt(h_g + h_o + 1.0)
        out[prec] = {"l1_rel": float(np.abs(h_g - h_o).sum() / max(h_o.sum(), 1e-300)),
                     "max_abs_z": float(z.max()),
                     "bins_differing": int((r["raw"][:, 1:-1] != ref["hist"]).sum()),
                     "detected_weight_rel": float(h_g.sum() / max(h_o.sum(), 1e-300) - 1.0)}
    cloud.close()
    return out


def precision_leg(ctx, stream, n):
    """cfg3 (tau = 109) at n packets on the FP32 and the plain FP64 GPU paths
    against the FP64 oracle's independent 1e7-packet spectrum
    (tests/golden/precision_cfg3.npz, another seed): merged-bin test, and the
    throughput of each path (both draw the same random numbers, so their errors
    are equal at equal packet counts)."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    g = np.load(os.path.join(ROOT, "tests", "golden", "precision_cfg3.npz"))
    n_ref = int(g["n_packets"])
    h_ref = g["hist"][0].astype(np.float64) / 2.0**32
    wl = W.cfg3(n_packets=n, r_ap=3.0 * W.MM, cone_alpha=0.5)
    cloud = pdv.Cloud(ctx, wl)
    out = {"packets_gpu": n, "packets_oracle": n_ref, "oracle_seed": int(g["seed"]),
           "gpu_seed": wl.seed, "tau_tot": float(g["tau_tot"])}
    for prec in ("fp32", "fp64"):
        pdv.simulate_spectrum(ctx, cloud, wl, precision=prec, n_packets=min(n, 100000))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = pdv.simulate_spectrum(ctx, cloud, wl, precision=prec)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        h = r["raw"][0, 1:-1].astype(np.float64) / 2.0**32
        out[prec] = dict(merged_bin_test(h, n, h_ref, n_ref), ms=ms,
                         packets_per_s=n / (ms / 1e3))
    cloud.close()
    out["throughput_ratio_fp32_over_fp64"] = out["fp32"]["packets_per_s"] / out["fp64"]["packets_per_s"]
    return out


def batch_leg(ctx, stream, scale):
    """cfg4's 256 parameter sets with their packet counts scaled by `scale`: one
    autotuned, graph-captured persistent launch, timed with CUDA events over 3
    launches; the same sets through the plain FP64 path; and four sets' tallies
    against the FP64 oracle on the same packets."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    sets = [w.replace(n_packets=max(1000, int(w.n_packets * scale))) for w in W.cfg4_sets()]
    clouds = [pdv.Cloud(ctx, w) for w in sets]
    reqs = [pdv.Request(c, w) for c, w in zip(clouds, sets)]
    def launches():
        pdv.pdv_simulate_batch(ctx.handle, [r.c for r in reqs])
        times = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pdv.pdv_simulate_batch(ctx.handle, [r.c for r in reqs])
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
        return statistics.median(times)

    ctx.set_tuning()                                   # the library's defaults
    t_untuned = launches()
    t0 = time.perf_counter()
    tuning = pdv.pdv_autotune(ctx.handle, [r.c for r in reqs])
    tune_s = time.perf_counter() - t0
    t = launches()
    scat = sum(int(r.result()["counters"][0][2]) for r in reqs)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for c, w in zip(clouds, sets):
        pdv.simulate_spectrum(ctx, c, w, precision="fp64", raw=False)
    b.record(stream)
    b.synchronize()
    f64 = a.elapsed_time(b) / 1e3
    check = []
    small = sorted(range(len(sets)), key=lambda i: sets[i].n_packets)[:4]
    for i in small:
        ref = O.simulate(sets[i], table=O.phase_table(sets[i]))
        got = reqs[i].result()["raw"][:, 1:-1]
        h_o, h_g = ref["hist"].astype(np.float64) / 2.0**32, got.astype(np.float64) / 2.0**32
        check.append({"set": i, "packets": sets[i].n_packets,
                      "bins_differing": int((got != ref["hist"]).sum()),
                      "max_abs_z": float((np.abs(h_g - h_o) / np.sqrt(h_g + h_o + 1.0)).max())})
    ctx.set_tuning()
    for c in clouds:
        c.close()
    return {"sets": len(sets), "packet_scale": scale,
            "packets_per_launch": int(sum(w.n_packets for w in sets)),
            "spectra_per_s": len(sets) / t, "ms_per_launch": 1e3 * t,
            "scatter_events_per_s": scat / t, "tuning": tuning, "autotune_s": tune_s,
            "ms_per_launch_untuned": 1e3 * t_untuned, "tuned_speedup": t_untuned / t,
            "fp64_plain_spectra_per_s": len(sets) / f64, "speedup_vs_fp64_plain": f64 / t,
            "oracle_same_packets": check}



def model_leg(ctx, stream, n=100_000):
    """Single-scattering spectra (Eq. 28) of n parameter sets and peak
    extraction (Eq. 29-35) of n noisy spectra, device-resident, CUDA-event
    timed; a few of each against the FP64 oracle (ss_peaks)."""
    import numpy as np
    import torch
    from oracle import ss_peaks as OS
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    nb, v_lo, v_hi, v_fs, k_c, x_lo, x_hi = 600, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5
    sets = W.model_sets(n, v_fs=v_fs)
    d_sets = torch.tensor(sets, device="cuda")
    d_spec = torch.empty(n * nb, dtype=torch.float64, device="cuda")
    d_pk = torch.empty(n * pdv.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    pdv.pdv_ss_spectrum(ctx.handle, d_sets, n, nb, v_lo, v_hi, d_spec, per_dv=True)
    d_in = (d_spec.view(n, nb) * torch.tensor(W.spectrum_noise((n, nb)), device="cuda")).contiguous()
    torch.cuda.synchronize()

    def timed(fn, reps=5):
        fn()
        ms, kms = [], []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            kms.append(ctx.stats()["last_model_ms"])
        return statistics.median(ms), statistics.median(kms)

    ss_ms, ss_k = timed(lambda: pdv.pdv_ss_spectrum(ctx.handle, d_sets, n, nb, v_lo, v_hi, d_spec,
                                                      per_dv=True))
    pk_simt_ms, pk_simt_k = timed(lambda: pdv.pdv_extract_peaks(ctx.handle, d_in, n, nb, v_lo, v_hi,
                                                                  v_fs, k_c, x_lo, x_hi, d_pk,
                                                                  simt=True))
    pk_simt = np.frombuffer(d_pk.cpu().numpy().tobytes(), pdv.PEAK_DTYPE).copy()
    pk_ms, pk_k = timed(lambda: pdv.pdv_extract_peaks(ctx.handle, d_in, n, nb, v_lo, v_hi, v_fs, k_c,
                                                        x_lo, x_hi, d_pk))
    spec = d_spec.view(n, nb)[:8].cpu().numpy()
    ss_err = max(float(np.max(np.abs(spec[i] - OS.ss_spectrum_bins(*sets[i][:3], nb, v_lo, v_hi,
                                                                     per_dv=True)) /
                         np.max(np.abs(spec[i])))) for i in range(8))
    pk = np.frombuffer(d_pk.cpu().numpy().tobytes(), pdv.PEAK_DTYPE)
    noisy = d_in[:8].cpu().numpy()
    beta_err = max(abs(pk["beta"][i] / OS.extract_peak(noisy[i], v_lo, v_hi, v_fs, k_c, x_lo, x_hi)["beta"]
                       - 1.0) for i in range(8))
    ok = (pk["status"] == pdv.PDV_PEAK_OK) & (pk_simt["status"] == pdv.PDV_PEAK_OK)
    paths_beta = float(np.max(np.abs(pk["beta"][ok] / pk_simt["beta"][ok] - 1.0))) if ok.any() else None
    return {"sets": n, "bins": nb, "k_c": k_c,
            "ss_spectra_per_s": n / (ss_ms / 1e3), "ss_kernel_ms": ss_k,
            "extract_spectra_per_s": n / (pk_ms / 1e3), "extract_kernel_ms": pk_k,
            "extract_path": "tensor cores (tcgen05, split TF32; the default)",
            "extract_simt_spectra_per_s": n / (pk_simt_ms / 1e3), "extract_simt_kernel_ms": pk_simt_k,
            "extract_paths_beta_max_rel": paths_beta,
            "oracle_check": {"ss_max_rel_to_peak": ss_err, "beta_max_rel": float(beta_err),
                             "sample": 8}}


def stepping_leg(ctx, stream, n=10_000_000):
    """The paper's layer stepping (1000 layers, acceptance-rejection angles) on
    the Fig. 4 cloud, n photons, CUDA-event timed; 500 photons against the
    oracle's stepping packet by packet (identical step counts)."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    wl = W.fig4(n_packets=n)
    table = O.phase_table(wl)
    cloud = pdv.Cloud(ctx, wl, table=table)
    pdv.simulate_spectrum(ctx, cloud, wl, n_packets=100000)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    st = ctx.stats()
    m = 500
    got = pdv.simulate_spectrum(ctx, cloud, wl, n_packets=m, packets=True)["packets"]
    ref = O.simulate(wl, n_packets=m, packets=True, table=table, spread_runs=0)["packets"]
    cloud.close()
    return {"photons": n, "layers": wl.n_layers, "seconds_per_spectrum": ms / 1e3,
            "photons_per_s": n / (ms / 1e3), "steps_per_s": st["last_steps"] / (st["last_transport_ms"] / 1e3),
            "vs_paper_gtx960": (n / (ms / 1e3)) / (1e7 / 500.0),
            "oracle_check": {"packets": m,
                             "same_step_counts": float(np.mean(got["n_events"] == ref["n_events"]))}}

# ----------------------------------------------------------------------- modes
def serving_run(ctx, seconds, rate):
    """Poisson stream of fit candidates through pdv_submit / pdv_poll against the
    oracle-generated target spectrum stored in tests/golden/serving_target.npz."""
    import numpy as np
    from paper_2012_00963_gb300 import serving
    from paper_2012_00963_gb300 import workloads as W
    g = np.load(os.path.join(ROOT, "tests", "golden", "serving_target.npz"))
    target = g["hist"][0].astype(np.float64) / 2.0**32
    probe = dict(r_ap=0.0, cone_alpha=math.pi / 2)       # every upward photon, as the target
    res = serving.run_sweep(ctx, target, int(g["n_packets"]), probe, duration=seconds, rate=rate,
                            keep_max_packets=150_000)
    hidden = {"beta": 6.0, "m0": 3.0 * W.MG_CM2, "d_m": 2.0 * W.UM, "tau0": float(g["tau_tot"])}
    out = serving.summary(res, hidden)
    out["oracle_same_packets"] = served_error(res.kept)
    out["capacity"] = serving_capacity(ctx, probe, rate)
    return out


def served_error(kept, n_each=4):
    """The first and the last `n_each` served requests of at most 1.5e5
    packets (the last ones are proposals of the fit, made while the stream was
    running) against the FP64 oracle on the same packets: bins that differ,
    the weight share in another bin, the largest per-bin z."""
    import numpy as np
    from oracle import oracle as O
    pick = kept[:n_each] + kept[max(n_each, len(kept) - n_each):]
    rows, differ, moved, tot, zmax = [], 0, 0.0, 0.0, 0.0
    for k, wl, raw in pick:
        ref = O.simulate(wl, spread_runs=0)["hist"]
        got = raw[:, 1:-1]
        h_o, h_g = ref.astype(np.float64) / 2.0**32, got.astype(np.float64) / 2.0**32
        differ += int((got != ref).sum())
        moved += float(np.abs(h_g - h_o).sum())
        tot += float(h_o.sum())
        zmax = max(zmax, float((np.abs(h_g - h_o) / np.sqrt(h_g + h_o + 1.0)).max()))
        rows.append({"arrival": int(k), "packets": int(wl.n_packets), "beta": float(wl.beta)})
    return {"requests": rows, "bins": sum(int(r[:, 1:-1].size) for _, _, r in pick),
            "bins_differing": differ, "l1_rel": moved / tot if tot else None, "max_abs_z": zmax}


def serving_capacity(ctx, probe, rate, n=64):
    """Spectra/s one GPU sustains on the served request mix (the first n
    arrivals of the stream) when each request runs alone on the FP32 path and
    on the plain FP64 path: both draw the same random numbers, so this is the
    comparison at equal spectrum error."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    arr = W.cfg5_arrivals()[:n]
    wls = [W.cfg5_request(a, **probe) for a in arr]
    clouds = [pdv.Cloud(ctx, w) for w in wls]
    out = {}
    for prec in ("fp32", "fp64"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat = []
        for c, w in zip(clouds, wls):
            t1 = time.perf_counter()
            pdv.simulate_spectrum(ctx, c, w, precision=prec, raw=False)   # blocking
            lat.append(1e3 * (time.perf_counter() - t1))
        out[prec + "_spectra_per_s"] = n / (time.perf_counter() - t0)
        # each request's latency when it runs alone (no queue): the path's own
        # service time, at equal spectrum error
        out[prec + "_alone_p50_ms"] = float(np.percentile(lat, 50))
        out[prec + "_alone_p99_ms"] = float(np.percentile(lat, 99))
    for c in clouds:
        c.close()
    out["ratio_fp32_over_fp64"] = out["fp32_spectra_per_s"] / out["fp64_spectra_per_s"]
    # a path whose capacity is below the stream's offered rate cannot keep its
    # queue bounded, whatever its latency alone
    out["offered_rate"] = rate
    out["fp64_sustains_offered_rate"] = bool(out["fp64_spectra_per_s"] >= rate)
    out["requests"] = n
    out["packets"] = int(sum(w.n_packets for w in wls))
    return out


def serve_mode(args):
    import torch
    from paper_2012_00963_gb300 import pdv
    torch.cuda.set_device(0)
    ctx = pdv.Context(0)
    clocks = Clocks(0)
    clocks.start()
    out = serving_run(ctx, args.serve_seconds, args.rate)
    clk = clocks.stop()
    ctx.close()
    line = {"mode": "serve", "metric": "p50/p99 request latency and spectra/s (served)",
            "unit": "ms", "rate_per_s": args.rate, "seconds": args.serve_seconds,
            "config": {"workload": "cfg5: Poisson stream of fit candidates (beta, m0, d), HG "
                                   "g=0.7 albedo 0.6, 400 bins 0-8000 m/s, 1e5-1e7 packets per "
                                   "request, every upward photon counted"},
            "clocks": clk}
    line.update(out)
    print(json.dumps(line))
    return 0


def batch_mode(args):
    """Batched launch of many parameter sets (cfg4) from one captured graph."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    sets = W.cfg4_sets(n_sets=args.sets, seed=4)
    clouds = [pdv.Cloud(ctx, w) for w in sets]
    reqs = [pdv.Request(c, w) for c, w in zip(clouds, sets)]
    tuning = pdv.pdv_autotune(ctx.handle, [r.c for r in reqs]) if args.autotune else None
    for _ in range(max(1, args.warmup)):
        pdv.pdv_simulate_batch(ctx.handle, [r.c for r in reqs])
    times, kern, scat, ev = [], [], 0, 0
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pdv.pdv_simulate_batch(ctx.handle, [r.c for r in reqs])
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        kern.append(ctx.stats()["last_transport_ms"])
        cnt = [r.result()["counters"][0] for r in reqs]
        scat += sum(int(c[2]) for c in cnt)
        ev += sum(int(c[1]) for c in cnt)
    clk = clocks.stop()
    tot = sum(times) / 1e3
    n_packets = sum(w.n_packets for w in sets)
    # the same sets through the plain FP64 path, one request at a time (the two
    # paths draw the same random numbers: equal spectrum error)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for c, w in zip(clouds, sets):
        pdv.simulate_spectrum(ctx, c, w, precision="fp64", raw=False)
    b.record(stream)
    b.synchronize()
    fp64_s = a.elapsed_time(b) / 1e3
    line = {"mode": "batch", "metric": "batched spectra/s", "value": len(sets) * args.steps / tot,
            "unit": "spectra/s", "scatter_events_per_s": scat / tot, "events_per_s": ev / tot,
            "ms_per_launch": 1e3 * tot / args.steps, "kernel_ms": statistics.mean(kern),
            "packets_per_launch": n_packets, "sets": len(sets), "tuning": tuning,
            "fp64_plain": {"spectra_per_s": len(sets) / fp64_s, "seconds": fp64_s},
            "speedup_vs_fp64_plain": (len(sets) * args.steps / tot) / (len(sets) / fp64_s),
            "gpu_launches_per_step": 2,
            "config": {"workload": "cfg4: %d sets, beta U(2,10), m0 logU(0.1,20) mg/cm^2, d "
                                   "logU(0.5,10) um Mie 3+9i, v_fs U(1.5,3) km/s, t U(1,4) us, "
                                   "packets logU(1e5,1e8), 400 bins" % len(sets)},
            "clocks": clk}
    for c in clouds:
        c.close()
    ctx.close()
    print(json.dumps(line))
    return 0


def precision_mode(args):
    """FP32 and FP64 GPU spectra of the heavy multiple-scattering cloud against
    the FP64 oracle's spectrum stored in tests/golden/precision_cfg3.npz."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    g = np.load(os.path.join(ROOT, "tests", "golden", "precision_cfg3.npz"))
    n_ref = int(g["n_packets"])
    h_ref = g["hist"][0].astype(np.float64) / 2.0**32
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    n = int(args.packets)
    wl = W.cfg3(n_packets=n, r_ap=3.0 * W.MM, cone_alpha=0.5)
    cloud = pdv.Cloud(ctx, wl)
    out = {}
    for prec in ("fp32", "fp64"):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = pdv.simulate_spectrum(ctx, cloud, wl, precision=prec)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        h = r["raw"][0, 1:-1].astype(np.float64) / 2.0**32
        c = pdv.counters_dict(r["counters"][0])
        out[prec] = dict(merged_bin_test(h, n, h_ref, n_ref), ms=ms, packets_per_s=n / (ms / 1e3),
                         scatter_events_per_s=c["scatters"] / (ms / 1e3))
    cloud.close()
    ctx.close()
    line = {"mode": "precision", "metric": "per-bin spectrum error vs the FP64 oracle, and "
            "throughput at equal error", "packets_gpu": n, "packets_oracle": n_ref,
            "tau_tot": float(g["tau_tot"]), "fp32": out["fp32"], "fp64": out["fp64"],
            "throughput_ratio_fp32_over_fp64": out["fp32"]["packets_per_s"] /
            out["fp64"]["packets_per_s"],
            "oracle_seed": int(g["seed"]), "gpu_seed": wl.seed,
            "note": "the oracle's spectrum draws another seed (independent samples); both GPU "
                    "paths draw the same random numbers, so at equal packet counts their "
                    "spectra (and errors against the oracle) are equal"}
    print(json.dumps(line))
    return 0


def model_counters():
    """Per-launch DRAM traffic of the spectrum-model and extraction kernels from
    the committed ncu summary, if it was taken on the current source."""
    p = os.path.join(ROOT, "profiles", "model_counters.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    src = open(os.path.join(ROOT, "paper_2012_00963_gb300", "csrc", "spectra.cu"), "rb").read()
    return d if d.get("source_hash") == hashlib.sha1(src).hexdigest()[:12] else None


def model_mode(args):
    """Single-scattering spectra (Eq. 28) of many parameter sets and main-peak
    extraction (Eq. 29-35) of as many noisy spectra, device-resident, timed
    with CUDA events; the same calls with host buffers end to end; the FP64
    oracle timed on a sample."""
    import numpy as np
    import torch
    from oracle import ss_peaks as OS
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    n, nb, v_lo, v_hi, v_fs, k_c, x_lo, x_hi = args.model_sets, 600, 0.0, 8000.0, 2000.0, 40, 1.02, 3.5
    sets = W.model_sets(n, v_fs=v_fs)
    d_sets = torch.tensor(sets, device="cuda")
    d_spec = torch.empty(n * nb, dtype=torch.float64, device="cuda")
    d_pk = torch.empty(n * pdv.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    flush = torch.empty(64 * 2**20, dtype=torch.float32, device="cuda")      # 256 MiB > L2

    def run_ss():
        pdv.pdv_ss_spectrum(ctx.handle, d_sets, n, nb, v_lo, v_hi, d_spec, per_dv=True)

    run_ss()
    d_in = (d_spec.view(n, nb) * torch.tensor(W.spectrum_noise((n, nb)), device="cuda")).contiguous()
    torch.cuda.synchronize()

    def run_pk():
        pdv.pdv_extract_peaks(ctx.handle, d_in, n, nb, v_lo, v_hi, v_fs, k_c, x_lo, x_hi, d_pk,
                              simt=args.extract_simt)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        wall, kern = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            wall.append(a.elapsed_time(b))
            kern.append(ctx.stats()["last_model_ms"])
        return statistics.mean(wall), statistics.mean(kern)

    clocks = Clocks(0)
    clocks.start()
    ss_ms, ss_kms = timed(run_ss)
    pk_ms, pk_kms = timed(run_pk)
    clk = clocks.stop()

    # end to end through the C ABI with host buffers (page-locked, as a serving
    # host would hold them: numpy views of pinned torch allocations)
    keep = []

    def pinned(a):
        t = torch.empty(a.nbytes, dtype=torch.uint8).pin_memory()
        keep.append(t)
        v = t.numpy().view(a.dtype).reshape(a.shape)
        v[...] = a
        return v

    sets_h = pinned(np.ascontiguousarray(sets).view(pdv.SS_SET_DTYPE).ravel())
    out_h = pinned(np.zeros(n * nb))
    spec_h = pinned(d_in.cpu().numpy())
    pk_h = pinned(np.zeros(n, dtype=pdv.PEAK_DTYPE))
    e2e = {}
    for name, fn in (("ss", lambda: pdv.pdv_ss_spectrum(ctx.handle, sets_h, n, nb, v_lo, v_hi, out_h,
                                                          per_dv=True)),
                     ("pk", lambda: pdv.pdv_extract_peaks(ctx.handle, spec_h, n, nb, v_lo, v_hi, v_fs,
                                                          k_c, x_lo, x_hi, pk_h,
                                                          simt=args.extract_simt))):
        fn()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        e2e[name] = (time.perf_counter() - t0) / args.steps
    ok = pk_h["status"] == pdv.PDV_PEAK_OK

    # the FP64 oracle on a sample (its inputs come from the oracle itself)
    m_ss, m_pk = 40, 200
    t0 = time.perf_counter()
    o_spec = [OS.ss_spectrum_bins(b, t, vf, nb, v_lo, v_hi, per_dv=True) for b, t, vf, _, _ in sets[:m_ss]]
    t_ss = time.perf_counter() - t0
    noisy = [o_spec[i % m_ss] * W.spectrum_noise(nb, seed=100 + i) for i in range(m_pk)]
    t0 = time.perf_counter()
    for sp in noisy:
        OS.extract_peak(sp, v_lo, v_hi, v_fs, k_c, x_lo, x_hi)
    t_pk = time.perf_counter() - t0

    prof = model_counters()
    xc = (v_lo + (np.arange(nb) + 0.5) * ((v_hi - v_lo) / nb)) / v_fs
    n_w = int(((xc >= x_lo) & (xc <= x_hi)).sum())
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    fma_peak = sm * 128 * 2.07e9                               # FP32 FMA lanes x max SM clock
    ss_bytes = n * nb * 8 + n * 40
    pk_bytes = n * nb * 8 + n * 48                              # FP64 spectra in, peak records out
    pk_flop = 2.0 * 2 * (k_c + 1) * (nb + n_w) * n             # two FP32 products, 2 flop / FMA
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    line = {
        "mode": "model",
        "metric": "single-scattering spectra/s (Eq. 28) and peak extractions/s (Eq. 29-35)",
        "ss_spectrum": {
            "value": n / (ss_ms / 1e3), "unit": "spectra/s", "ms_per_call": ss_ms, "kernel_ms": ss_kms,
            "bins_per_s": n * nb / (ss_kms / 1e3), "gpu_launches": 2,
            "roofline": {"bound": "hbm", "achieved": ss_bytes / (ss_kms / 1e3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": ss_bytes / (ss_kms / 1e3) / 1e9 / hbm,
                         "traffic": prof["k_ss_bins"]["dram_bytes_per_launch"] if prof else None,
                         "kernel": "k_ss_bins", "peak_source": "measured"},
            "e2e": {"value": n / e2e["ss"], "unit": "spectra/s", "h2d_bytes_per_step": n * 40,
                    "d2h_bytes_per_step": n * nb * 8},
            "cpu_baseline": {"value": m_ss / t_ss, "unit": "spectra/s", "cores": 1, "kind": "oracle",
                             "sample": "%d sets, composite Gauss-Legendre per bin" % m_ss}},
        "extract_peaks": {
            "value": n / (pk_ms / 1e3), "unit": "spectra/s", "ms_per_call": pk_ms, "kernel_ms": pk_kms,
            "gpu_launches": 3, "ok_fraction": float(ok.mean()),
            "path": ("FP32 FMA on the CUDA cores" if args.extract_simt
                     else "tensor cores (tcgen05, split TF32)"),
            # the CUDA-core kernel is bound by FP32 FMA issue; the tensor-core
            # kernel's floor is reading the FP64 spectra from HBM
            "roofline": ({"bound": "alu", "achieved": pk_flop / (pk_kms / 1e3) / 1e12,
                          "peak": 2 * fma_peak / 1e12, "unit": "TFLOP/s",
                          "frac": pk_flop / (pk_kms / 1e3) / (2 * fma_peak),
                          "traffic": prof["k_extract_tiled"]["dram_bytes_per_launch"] if prof else None,
                          "kernel": "k_extract_tiled",
                          "peak_source": "%d SM x 128 FP32 lanes x 2070 MHz x 2 flop" % sm,
                          "algorithmic_flop_per_spectrum": pk_flop / n}
                         if args.extract_simt else
                         {"bound": "hbm", "achieved": pk_bytes / (pk_kms / 1e3) / 1e9, "peak": hbm,
                          "unit": "GB/s", "frac": pk_bytes / (pk_kms / 1e3) / 1e9 / hbm,
                          "traffic": (prof["k_extract_tc"]["dram_bytes_per_launch"] * n / 1e5
                                      if prof and "k_extract_tc" in prof else None),
                          "kernel": "k_extract_tc", "peak_source": "measured",
                          "algorithmic_bytes_per_spectrum": pk_bytes / n,
                          "tensor_flop_per_spectrum": 3 * pk_flop / n}),
            "e2e": {"value": n / e2e["pk"], "unit": "spectra/s", "h2d_bytes_per_step": n * nb * 8,
                    "d2h_bytes_per_step": n * pdv.PEAK_DTYPE.itemsize},
            "cpu_baseline": {"value": m_pk / t_pk, "unit": "spectra/s", "cores": 1, "kind": "oracle",
                             "sample": "%d noisy spectra, numpy FFT + Newton" % m_pk}},
        "steps": args.steps, "warmup": max(3, args.warmup), "dtype": "f32",
        "data": "synthetic (seeded parameter sets; spectra with 2% multiplicative noise)",
        "config": {"workload": "%d sets beta U(2,12), tau0 logU(2,60), v_fs 2000 m/s; %d bins over "
                               "0-8000 m/s per dv; extraction k_c=%d, window x in [%.2f, %.1f]"
                               % (n, nb, k_c, x_lo, x_hi),
                   "l2": "flushed between steps (256 MiB write)"},
        "clocks": clk,
    }
    ctx.close()
    print(json.dumps(line))
    return 0


def extract_mc_mode(args):
    """The study of Figs. 13-15 (Section III.B): Monte Carlo spectra of the two
    clouds quoted there (tau0 = 23.4 and 8.6) over a range of beta, each
    reduced by the peak extraction; the single-scattering prediction (Eq. 31,
    Eq. 34) beside them, and the extraction of the model spectrum itself."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    betas = (4.0, 6.0, 8.0, 10.0, 12.0, 14.0)
    rows = []
    for ci, c in enumerate(W.FIG13_CLOUDS):
        for beta in betas:
            wl = W.fig13(ci, beta, n_packets=int(args.packets) if args.packets != 1e8 else 10_000_000)
            cloud = pdv.Cloud(ctx, wl)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)
            b.record(stream)
            b.synchronize()
            info = cloud.info()
            cloud.close()
            span = (wl.v_hi - wl.v_lo) / wl.v_fs
            k_c = min(int(math.ceil(1.25 * beta * span)), wl.n_bins // 2 - 1)
            pk = pdv.extract_peaks(ctx, r["spectrum"][0], wl.v_lo, wl.v_hi, wl.v_fs, k_c, 1.02,
                                   3.5)[0]
            ss = pdv.ss_spectrum(ctx, [(beta, c["tau0_paper"], wl.v_fs, 0.0, 1.0)], wl.n_bins,
                                 wl.v_lo, wl.v_hi, per_dv=True)
            pk_ss = pdv.extract_peaks(ctx, ss[0], wl.v_lo, wl.v_hi, wl.v_fs, k_c, 1.02, 3.5)[0]
            cnt = pdv.counters_dict(r["counters"][0])
            rows.append({
                "cloud": c["label"], "beta": beta, "tau0_paper": c["tau0_paper"],
                "tau_ext_cloud": info["tau_tot"], "k_c": k_c, "mc_ms": a.elapsed_time(b),
                "detected_fraction": cnt["w_detected"] / 2.0**32 / wl.n_packets,
                "theory": {"x_peak": 1.0 + math.log(c["tau0_paper"]) / beta, "curvature": -beta * beta},
                "mc": {"x_peak": float(pk["x_peak"]), "curvature": float(pk["curvature"]),
                       "beta": float(pk["beta"]), "tau0": float(pk["tau0"]), "status": int(pk["status"])},
                "ss_model": {"x_peak": float(pk_ss["x_peak"]), "beta": float(pk_ss["beta"]),
                             "tau0": float(pk_ss["tau0"]), "status": int(pk_ss["status"])}})
    ctx.close()
    print(json.dumps({"mode": "extract-mc",
                      "metric": "peak position and relative curvature of Monte Carlo spectra vs "
                                "the single-scattering relations (Eq. 31, Eq. 34)",
                      "config": {"workload": "Figs. 13-15 clouds: m0 20 / 10 mg/cm^2, d_m 1.5 / 2.0 "
                                             "um, sigma 0.5, Mie 3+9i, every upward photon, 1200 "
                                             "bins 0-8000 m/s, t = 1 us"},
                      "rows": rows}))
    return 0


def trends_mode(args):
    """Section III.A on this Monte Carlo: one parameter at a time around a
    base cloud (beta 8, d_m 1.5 um, sigma 0.5, 10 mg/cm^2, Mie 3+9i, every
    upward photon), the main peak position (extraction pipeline, window
    x >= 1.02) and the share of the detected weight below v_fs, where the
    free-surface echo lands."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    ctx = pdv.Context(0, stream=torch.cuda.current_stream().cuda_stream)
    n = int(args.packets) if args.packets != 1e8 else 10_000_000
    base = W.fig6(1, n_packets=n, m0=10.0 * W.MG_CM2, n_bins=800, seed=31)
    sweeps = {"beta": [("beta", v, {"beta": v}) for v in (4.0, 8.0, 12.0)],
              "d_m_um": [("d_m_um", v, {"d_m": v * W.UM}) for v in (1.0, 2.0, 4.0)],
              "m0_mg_cm2": [("m0_mg_cm2", v, {"m0": v * W.MG_CM2}) for v in (2.0, 5.0, 10.0, 20.0)]}
    out = {}
    for key, cases in sweeps.items():
        rows = []
        for _, v, kw in cases:
            wl = base.replace(**kw)
            cloud = pdv.Cloud(ctx, wl)
            r = pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)
            tau = cloud.info()["tau_tot"]
            cloud.close()
            sp = r["spectrum"][0]
            vc = wl.v_lo + (np.arange(wl.n_bins) + 0.5) * (wl.v_hi - wl.v_lo) / wl.n_bins
            span = (wl.v_hi - wl.v_lo) / wl.v_fs
            k_c = min(int(math.ceil(1.25 * wl.beta * span)), wl.n_bins // 2 - 1)
            pk = pdv.extract_peaks(ctx, sp, wl.v_lo, wl.v_hi, wl.v_fs, k_c, 1.02, 6.0)[0]
            rows.append({key: v, "tau_ext": tau, "x_peak": float(pk["x_peak"]),
                         "status": int(pk["status"]),
                         "share_below_v_fs": float(sp[vc < wl.v_fs].sum() / sp.sum())})
        out[key] = rows
    ctx.close()
    print(json.dumps({"mode": "trends",
                      "metric": "main-peak position and free-surface share of Monte Carlo spectra "
                                "against beta, particle size and area mass (Section III.A)",
                      "config": {"workload": "base: tin, beta 8, d_m 1.5 um, sigma 0.5, 10 mg/cm^2, "
                                             "Mie 3+9i, every upward photon, 800 bins 0-8000 m/s, "
                                             "t = 1 us, %d packets per case" % n},
                      "sweeps": out}))
    return 0


def fig6_mode(args):
    """Section II.D, Fig. 6, cases 1 and 2: the same cloud scattering by its
    Mie phase function and isotropically (with the same Mie extinction and
    albedo), every upward photon counted. For each case: the main peak (the
    extraction pipeline), the detected fraction and the mean apparent
    velocity; between them: the L1 distance of the unit-area spectra, split at
    the Mie case's peak into the part below (the low-velocity, dense part of
    the cloud) and above."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    out, spec = {}, {}
    for case in (1, 2):
        wl = W.fig6(case, n_packets=int(args.packets) if args.packets != 1e8 else 10_000_000)
        cloud = pdv.Cloud(ctx, wl)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)
        b.record(stream)
        b.synchronize()
        cloud.close()
        s = r["spectrum"][0]
        vc = wl.v_lo + (np.arange(wl.n_bins) + 0.5) * (wl.v_hi - wl.v_lo) / wl.n_bins
        span = (wl.v_hi - wl.v_lo) / wl.v_fs
        k_c = min(int(math.ceil(1.25 * wl.beta * span)), wl.n_bins // 2 - 1)
        pk = pdv.extract_peaks(ctx, s, wl.v_lo, wl.v_hi, wl.v_fs, k_c, 1.02, 3.5)[0]
        c = pdv.counters_dict(r["counters"][0])
        spec[case] = (s, vc)
        out["case%d" % case] = {"phase": "Mie" if case == 1 else "isotropic (Mie extinction and albedo)",
                                "x_peak": float(pk["x_peak"]), "status": int(pk["status"]),
                                "detected_fraction": c["w_detected"] / 2.0**32 / wl.n_packets,
                                "mean_v_app_detected": float((s * vc).sum() / s.sum()),
                                "mc_ms": a.elapsed_time(b)}
    (s1, vc), (s2, _) = spec[1], spec[2]
    d = np.abs(s1 / s1.sum() - s2 / s2.sum())
    v_split = out["case1"]["x_peak"] * W.fig6(1).v_fs
    ctx.close()
    print(json.dumps({"mode": "fig6",
                      "metric": "Mie vs isotropic scattering on the Fig. 6 cloud: peaks, detected "
                                "fraction, and where the unit-area spectra differ",
                      "config": {"workload": "Fig. 6 cloud: tin, m0 10.7 mg/cm^2, d_m 1.5 um, sigma 0.5, "
                                             "beta 8, Mie 3+9i vs isotropic, every upward photon, "
                                             "600 bins 0-8000 m/s, t = 1 us, 1e7 packets"},
                      "case1": out["case1"], "case2": out["case2"],
                      "shape_l1": float(d.sum()), "shape_l1_below_case1_peak": float(d[vc < v_split].sum()),
                      "shape_l1_above_case1_peak": float(d[vc >= v_split].sum())}))
    return 0


def implicit_mode(args):
    """Analog absorption (Eq. 11) against implicit capture with Russian
    roulette on the 50-snapshot log-normal Mie cloud: K independent seeds per
    scheme give each bin's mean and variance; the figure of merit is the
    spectrum's squared signal-to-noise per second of transport,
    (sum_b mean_b^2 / sum_b var_b) / T. chi2_per_bin compares the two schemes'
    means (about 1 when they estimate the same spectrum)."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    ctx = pdv.Context(0)
    n = int(args.packets) if args.packets != 1e8 else 10_000_000
    K = max(int(args.steps), 4)
    base = W.cfg2(n_packets=n)
    cloud = pdv.Cloud(ctx, base)
    res = {}
    for name, imp in (("analog", False), ("implicit", True)):
        wl0 = base.replace(implicit_capture=imp)
        pdv.simulate_spectrum(ctx, cloud, wl0.replace(seed=999, n_packets=min(n, 1_000_000)))
        specs, ms, ev, det = [], [], [], []
        for k in range(K):
            r = pdv.simulate_spectrum(ctx, cloud, wl0.replace(seed=1000 + k))
            st = ctx.stats()
            specs.append(r["spectrum"])
            ms.append(st["last_transport_ms"])
            c = pdv.counters_dict(r["counters"][0])
            ev.append(c["events"])
            det.append(c["w_detected"] / 2.0**32 / n)
        S = np.array(specs)
        mean, var = S.mean(axis=0), S.var(axis=0, ddof=1)
        t = float(np.median(ms))
        snr2 = float((mean**2).sum() / var.sum())
        res[name] = {"transport_ms": t, "events_per_packet": float(np.mean(ev)) / n,
                     "detected_fraction_t0": float(np.mean(det)),
                     "relative_noise": float(np.sqrt(1.0 / snr2)), "fom_per_s": snr2 / (t * 1e-3),
                     "mean": mean, "var": var}
    a, b = res["analog"], res["implicit"]
    chi2 = float(((a["mean"] - b["mean"])**2 / ((a["var"] + b["var"]) / K + 1e-300))[
        (a["var"] + b["var"]) > 0].mean())
    cloud.close()
    ctx.close()
    for v in res.values():
        del v["mean"], v["var"]
    print(json.dumps({"mode": "implicit",
                      "metric": "squared signal-to-noise of the spectrum per second of transport, "
                                "analog (Eq. 11) vs implicit capture + Russian roulette",
                      "config": {"workload": "cfg2: log-normal Mie cloud d_m=3um sigma=0.5 m=3+9i, "
                                             "5 mg/cm^2 tin, beta=5, 50 snapshots 0.5-5us, %d packets, "
                                             "%d seeds per scheme, 600 bins" % (n, K)},
                      "analog": a, "implicit": b, "fom_ratio_implicit_over_analog":
                      b["fom_per_s"] / a["fom_per_s"], "chi2_per_bin_between_means": chi2}))
    return 0


def fig12_mode(args):
    """The single-scattering model beside the Monte Carlo (Section III.B,
    Fig. 12): for each area mass, the Monte Carlo spectrum of the cloud and the
    model spectrum of Eq. 28 with tau0 = g_back tau_ext (the cloud's extinction
    depth; g_back the paper's 0.67, and Eq. 25 evaluated for this cloud's own
    scattering law), compared by shape (L1 distance of the unit-area spectra:
    0 equal, 2 disjoint) and by main-peak position (the extraction pipeline on
    all of them, Eq. 31 beside them); and the time of one spectrum by each."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    g_back, beta, rows = 0.67, 10.0, []
    for m0 in W.FIG12_MASSES:
        wl = W.fig12(m0, n_packets=int(args.packets) if args.packets != 1e8 else 10_000_000)
        cloud = pdv.Cloud(ctx, wl)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mc = pdv.simulate_spectrum(ctx, cloud, wl, per_dv=True)["spectrum"][0]
        b.record(stream)
        b.synchronize()
        mc_ms = a.elapsed_time(b)
        tau_ext = cloud.info()["tau_tot"]
        cloud.close()
        # Eq. 25 for this cloud's own scattering law: g_back = (K_back + K_abs) / K_ext,
        # with K_back the scattering into the backward hemisphere of the phase table
        th, pt, _, albedo = pdv.phase_table(ctx, wl)
        w = pt * np.sin(th)
        cum = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(th))])
        back = 1.0 - np.interp(0.5 * math.pi, th, cum) / cum[-1]
        g_own = albedo * back + (1.0 - albedo)
        models = {}
        for name, g in (("paper_g_back", g_back), ("own_g_back", g_own)):
            tau0 = g * tau_ext
            a.record(stream)
            ss = pdv.ss_spectrum(ctx, [(beta, tau0, wl.v_fs, 0.0, 1.0)], wl.n_bins, wl.v_lo,
                                 wl.v_hi, per_dv=True)[0]
            b.record(stream)
            b.synchronize()
            models[name] = (g, tau0, ss, a.elapsed_time(b))
        span = (wl.v_hi - wl.v_lo) / wl.v_fs
        k_c = min(int(math.ceil(1.25 * beta * span)), wl.n_bins // 2 - 1)
        pk = pdv.extract_peaks(ctx, np.stack([mc] + [m[2] for m in models.values()]), wl.v_lo,
                               wl.v_hi, wl.v_fs, k_c, 1.02, 3.5)
        row = {"m0_mg_cm2": m0, "tau_ext": tau_ext, "x_peak_mc": float(pk[0]["x_peak"]),
               "status_mc": int(pk[0]["status"]), "mc_ms": mc_ms}
        for i, (name, (g, tau0, ss, ms)) in enumerate(models.items()):
            l1 = float(np.abs(mc / mc.sum() - ss / ss.sum()).sum()) if mc.sum() > 0 and ss.sum() > 0 else None
            row[name] = {"g_back": g, "tau0": tau0, "x_peak_eq31": 1.0 + math.log(tau0) / beta,
                         "x_peak_model": float(pk[1 + i]["x_peak"]),
                         "status_model": int(pk[1 + i]["status"]), "shape_l1": l1, "model_ms": ms}
        rows.append(row)
    ctx.close()
    print(json.dumps({"mode": "fig12",
                      "metric": "shape and main-peak position of the single-scattering model vs the "
                                "Monte Carlo spectrum (Eq. 28, Eq. 31)",
                      "config": {"workload": "Fig. 12 clouds: beta 10, d_m 1.5 um, sigma 0.5, Mie 3+9i, "
                                             "m0 5-40 mg/cm^2, every upward photon, 1200 bins "
                                             "0-8000 m/s, t = 1 us; model with g_back = 0.67 and with "
                                             "the cloud's own Eq. 25 value"},
                      "rows": rows}))
    return 0


def stepping_mode(args):
    """The paper's own scheme (1000 layers, acceptance-rejection angles) on the
    workload its timings are quoted on (Fig. 4: 1e7 photons), against the exact
    free-path scheme on the same cloud, and the oracle's stepping on a sample."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    n = int(args.packets) if args.packets != 1e8 else 10_000_000
    wl = W.fig4(n_packets=n)
    cloud = pdv.Cloud(ctx, wl)
    out = {}
    clocks = Clocks(0)
    clocks.start()
    for name, w in (("stepping", wl), ("exact", wl.replace(n_layers=0))):
        pdv.simulate_spectrum(ctx, cloud, w, n_packets=min(n, 100000))      # warm-up
        ms, kms = [], []
        for _ in range(max(1, args.steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = pdv.simulate_spectrum(ctx, cloud, w, per_dv=True)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            kms.append(ctx.stats()["last_transport_ms"])
        c = pdv.counters_dict(r["counters"][0])
        st = ctx.stats()
        hist = r["raw"][0, 1:-1].astype(np.float64) / 2.0**32
        vc = (np.arange(wl.n_bins) + 0.5) * (wl.v_hi - wl.v_lo) / wl.n_bins + wl.v_lo
        out[name] = {"ms": statistics.mean(ms), "kernel_ms": statistics.mean(kms),
                     "photons_per_s": n / (statistics.mean(ms) / 1e3),
                     "scatter_events_per_s": c["scatters"] / (statistics.mean(ms) / 1e3),
                     "events": c["events"], "scatters": c["scatters"],
                     "detected_fraction": c["w_detected"] / 2.0**32 / n,
                     "mean_v_app_detected": float((hist * vc).sum() / hist.sum()),
                     "hist": hist}
        if name == "stepping":
            out[name]["steps"] = st["last_steps"]
            out[name]["steps_per_s"] = st["last_steps"] / (statistics.mean(kms) / 1e3)
    clk = clocks.stop()
    issue_meas = pdv.pdv_measure_issue_rate(ctx.handle, 0.2)        # after the timed region
    info = cloud.info()
    cloud.close()
    ctx.close()
    h_s, h_e = out["stepping"].pop("hist"), out["exact"].pop("hist")
    sel = (h_s + h_e) > 50
    chi2 = float(np.mean((h_s[sel] - h_e[sel]) ** 2 / (h_s[sel] + h_e[sel])))
    # the oracle's stepping on a sample of the same workload
    m = 400
    t0 = time.perf_counter()
    O.simulate(wl, n_packets=m, n_threads=os.cpu_count())
    t_cpu = time.perf_counter() - t0
    paper_photons_per_s = 1e7 / 500.0                  # GTX960, Section II.D
    # issue-rate roofline of the stepping kernel: algorithmic work per step is
    # one Philox4x32-10 call (64), the Bernoulli exponential (10), the layer
    # mass of Eq. 20 (16) and the step itself (20): 110 thread-instructions
    a_step = 110.0
    sm = torch.cuda.get_device_properties(0).multi_processor_count if torch.cuda.is_available() else 152
    issue_peak = sm * 4 * 32 * 2.07e9
    achieved = a_step * out["stepping"]["steps_per_s"]
    prof = None
    pp = os.path.join(ROOT, "profiles", "transport_step_counters.json")
    if os.path.exists(pp):
        d = json.load(open(pp))
        src = open(os.path.join(ROOT, "paper_2012_00963_gb300", "csrc", "stepping.cu"), "rb").read()
        if d.get("source_hash") == hashlib.sha1(src).hexdigest()[:12]:
            prof = d
    line = {
        "mode": "stepping",
        "metric": "photons/s of the paper's layer-stepping scheme (1000 layers), 1e7-photon spectrum",
        "value": out["stepping"]["photons_per_s"], "unit": "photons/s",
        "vs_paper_gtx960": out["stepping"]["photons_per_s"] / paper_photons_per_s,
        "seconds_per_1e7_photon_spectrum": 1e7 / out["stepping"]["photons_per_s"],
        "stepping": out["stepping"], "exact": out["exact"],
        "exact_over_stepping_speed": out["exact"]["photons_per_s"] / out["stepping"]["photons_per_s"],
        "spectrum_chi2_per_bin_stepping_vs_exact": chi2,
        "mean_v_app_shift_m_s": out["stepping"]["mean_v_app_detected"] - out["exact"]["mean_v_app_detected"],
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": issue_peak / 1e9,
                     "unit": "Ginst/s", "frac": achieved / issue_peak,
                     "traffic": prof["dram_bytes_per_step"] * out["stepping"]["steps"] if prof else None,
                     "kernel": "k_transport_step", "algo_inst_per_step": a_step,
                     "peak_basis": "%d SM x 4 schedulers x 32 lanes x 2070 MHz (issue rate)" % sm,
                     "peak_measured": issue_meas / 1e9, "frac_of_measured": achieved / issue_meas},
        "gpu_launches": 1,
        "tau_tot": info["tau_tot"], "dtype": "f32", "data": "synthetic (seeded)",
        "cpu_baseline": {"value": m / t_cpu, "unit": "photons/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": "%d photons of the same workload, layer stepping" % m},
        "config": {"workload": "Fig. 4 cloud: tin, beta 10, d_m 1.5 um, sigma 0.5, 20 mg/cm^2, Mie 3+9i "
                               "at 1550 nm, every upward photon, %d photons, 1000 layers, 600 bins" % n},
        "clocks": clk}
    print(json.dumps(line))
    return 0


def spectrogram_mode(args):
    """A v-t spectrogram of the 50-snapshot workload's cloud at --times
    snapshot times (one transport serves every time), device-resident."""
    import numpy as np
    import torch
    from paper_2012_00963_gb300 import pdv
    from paper_2012_00963_gb300 import spectrogram as S
    from paper_2012_00963_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = pdv.Context(0, stream=stream.cuda_stream)
    n = int(args.packets)
    t = np.linspace(0.5e-6, 5e-6, args.times)
    wl = W.cfg2(n_packets=n)
    cloud = pdv.Cloud(ctx, wl)
    S.spectrogram(ctx, cloud, wl, t[:4])                        # warm-up
    clocks = Clocks(0)
    clocks.start()
    ms, kms = [], []
    for _ in range(max(1, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sg = S.spectrogram(ctx, cloud, wl, t)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        kms.append(ctx.stats()["last_transport_ms"])
    clk = clocks.stop()
    c = pdv.counters_dict(sg["counters"][0])
    if args.out:
        S.write_pgm(args.out, sg["image"])
    cloud.close()
    ctx.close()
    mean = statistics.mean(ms)
    print(json.dumps({
        "mode": "spectrogram", "metric": "spectra/s of a v-t spectrogram (one transport, every time)",
        "value": args.times / (mean / 1e3), "unit": "spectra/s", "ms_per_image": mean,
        "kernel_ms": statistics.mean(kms), "scatter_events_per_s": c["scatters"] / (mean / 1e3),
        "times": args.times, "packets": n, "gpu_launches": 2, "dtype": "f32",
        "config": {"workload": "cfg2 cloud (log-normal Mie 3+9i, 5 mg/cm^2, beta 5), %d snapshot times "
                               "0.5-5 us, %d packets, 600 bins, aperture 1 mm / 0.1 rad" % (args.times, n)},
        "clocks": clk}))
    return 0


def cpu_baseline_mode(args):
    """The FP64 CPU oracle timed on this machine's host cores, with one thread
    and with all of them: the cfg1 workload on 1e6 packets and the heavy
    multiple-scattering cfg3 cloud (tau = 109) on 1e7 packets. Events/s,
    scatter events/s and spectra/s per run; no GPU is used."""
    from oracle import oracle as O
    from paper_2012_00963_gb300 import workloads as W
    cores = os.cpu_count() or 1
    out = {}
    for name, wl, n_all, n_one in (
            ("cfg1", W.cfg1(), 1_000_000, 1_000_000),
            ("cfg3", W.cfg3(r_ap=3.0 * W.MM, cone_alpha=0.5), 10_000_000, 10_000_000)):
        table = O.phase_table(wl)
        row = {"workload": wl.name, "snapshots": len(wl.t_snap)}
        for key, threads, n in (("all_cores", cores, n_all), ("one_thread", 1, n_one)):
            t0 = time.perf_counter()
            r = O.simulate(wl, n_threads=threads, n_packets=n, table=table)
            dt = time.perf_counter() - t0
            c = r["counters"][0]
            row[key] = {"threads": threads, "packets": n, "seconds": dt,
                        "events_per_s": int(c[1]) / dt, "scatter_events_per_s": int(c[2]) / dt,
                        "packets_per_s": n / dt,
                        "spectra_per_s": len(wl.t_snap) * (n / wl.n_packets) / dt}
        out[name] = row
    line = {"mode": "cpu-baseline", "metric": "FP64 oracle events/s and spectra/s on the host cores",
            "kind": "oracle", "cores": cores, "cfg1": out["cfg1"], "cfg3": out["cfg3"],
            "note": "spectra/s counts whole spectra of each workload's full packet count "
                    "(cfg1 1e6, cfg3 1e9 packets)"}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.mode == "serve":
        return serve_mode(args)
    if args.mode == "batch":
        return batch_mode(args)
    if args.mode == "precision":
        return precision_mode(args)
    if args.mode == "model":
        return model_mode(args)
    if args.mode == "extract-mc":
        return extract_mc_mode(args)
    if args.mode == "stepping":
        return stepping_mode(args)
    if args.mode == "trends":
        return trends_mode(args)
    if args.mode == "fig6":
        return fig6_mode(args)
    if args.mode == "fig12":
        return fig12_mode(args)
    if args.mode == "implicit":
        return implicit_mode(args)
    if args.mode == "cpu-baseline":
        return cpu_baseline_mode(args)
    if args.mode == "spectrogram":
        return spectrogram_mode(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
