"""Serving-side parameter sweep over the library's continuous-batching loop.

A stream of spectrum requests arrives as a Poisson process. Each request is a
candidate (beta, m0, d) of a fit to a target spectrum (Section III: the
spectrum is fixed mainly by beta and the optical depth tau0, so m0 and d are
degenerate along m0/d). Requests are admitted with pdv_submit while others are
running and finish through pdv_poll; the driver records every request's
latency (submit to completion) and keeps the best candidate.

The library does all Monte Carlo work on the GPU; this module only proposes
parameters, marshals requests and scores finished spectra (a chi-square
between two histograms on the host).
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import pdv
from . import workloads as W


@dataclass
class SweepResult:
    latencies_ms: List[float] = field(default_factory=list)
    completed: int = 0
    rejected: int = 0
    wall_s: float = 0.0
    best: dict = field(default_factory=dict)
    submitted: int = 0
    records: List[dict] = field(default_factory=list)
    kept: List[tuple] = field(default_factory=list)    # (arrival index, workload, raw tally)


def chi2(h_c, n_c, h_t, n_t, min_counts=10.0):
    """Chi-square per bin between a candidate's and the target's weight
    histograms (packet units) normalised per launched packet, over the bins
    where the target holds at least `min_counts`; the variance of both sides
    is taken from the target's rate (the null hypothesis)."""
    s_c, s_t = h_c / n_c, h_t / n_t
    sel = h_t >= min_counts
    var = s_t[sel] * (1.0 / n_c + 1.0 / n_t)
    return float(np.sum((s_c[sel] - s_t[sel]) ** 2 / var)), int(sel.sum())


def surrogate_estimate(records, min_packets=1_000_000, keep=0.4, min_points=12):
    """Vertex of a least-squares quadratic in (log beta, log tau0) fitted to
    chi^2/dof of the best-scoring well-sampled candidates; None when fewer than
    `min_points` qualify or the fitted bowl is not convex. Beta and tau0 are the
    two parameters a single spectrum fixes (Eq. 35)."""
    r = [x for x in records if x["n"] >= min_packets]
    if len(r) < min_points:
        return None
    r.sort(key=lambda x: x["chi2"])
    r = r[:max(min_points, int(len(r) * keep))]
    X = np.log([x["beta"] for x in r])
    Y = np.log([x["tau0"] for x in r])
    Z = np.array([x["chi2"] for x in r])
    A = np.stack([np.ones_like(X), X, Y, X * X, Y * Y, X * Y], axis=1)
    (a, b, c, d, e, f), *_ = np.linalg.lstsq(A, Z, rcond=None)
    H = np.array([[2 * d, f], [f, 2 * e]])
    if np.any(np.linalg.eigvalsh(H) <= 0):
        return None
    x0, y0 = np.linalg.solve(H, [-b, -c])
    if not (X.min() - 1 <= x0 <= X.max() + 1 and Y.min() - 1 <= y0 <= Y.max() + 1):
        return None
    return {"beta": float(math.exp(x0)), "tau0": float(math.exp(y0)), "points": len(r)}


def run_sweep(ctx: pdv.Context, target_hist, target_packets, probe: dict, duration: float = 60.0,
              rate: float = 200.0, seed: int = 5, n_min: float = 1e5, n_max: float = 1e7,
              explore: float = 0.2, poll_us: int = 200,
              min_best_packets: int = 1_000_000, lag: int = 20,
              keep_max_packets: int = 0) -> SweepResult:
    """Submit the Poisson stream of candidates and score them as they finish.
    The candidate proposed at arrival k is computed only from the results of
    arrivals 0 .. k - lag, taken in arrival order, so the candidate sequence
    and the recovered parameters do not depend on the order in which requests
    complete (at 200 requests/s a lag of 20 is 0.1 s, far above the serving
    latency, so the submitter almost never waits for it). Requests of at most
    `keep_max_packets` packets keep their workload and raw tally in
    `SweepResult.kept`, so that a caller can check served results."""
    arrivals = W.cfg5_arrivals(rate=rate, duration=duration, seed=seed, n_min=n_min,
                               n_max=n_max)
    rng = np.random.default_rng(seed + 1)
    res = SweepResult()
    lock = threading.Lock()
    pending = {}            # ticket -> (request, cloud, t_submit, params, arrival index, workload)
    done = {}               # arrival index -> record (None: no scored bins)
    target = np.asarray(target_hist, np.float64)
    done_submitting = threading.Event()
    surrogate_center = {}
    best = {"chi2": math.inf}
    folded = 0              # arrivals 0 .. folded - 1 are folded into `best` and `prefix`
    prefix = []             # their records, in arrival order

    def poller():
        while True:
            with lock:
                items = list(pending.items())
            if not items:
                if done_submitting.is_set():
                    return
                time.sleep(0.0002)
                continue
            for t, (req, cloud, t0, params, k, wl) in items:
                st = pdv.pdv_poll(ctx.handle, t, poll_us // max(len(items), 1))
                if st != pdv.PDV_OK:
                    continue
                t1 = time.perf_counter()
                h = req.raw[0, 1:-1].astype(np.float64) / 2.0**32
                c2, dof = chi2(h, req.c.n_packets, target, target_packets)
                tau0 = cloud.info()["tau_tot"]
                rec = (dict(beta=params["beta"], tau0=tau0, m0=params["m0"], d_m=params["d_m"],
                            chi2=c2 / dof, n=int(req.c.n_packets)) if dof else None)
                with lock:
                    del pending[t]
                    res.latencies_ms.append(1e3 * (t1 - t0))
                    res.completed += 1
                    done[k] = rec
                    if wl.n_packets <= keep_max_packets:
                        res.kept.append((k, wl, req.raw.copy()))

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    clouds = []
    t_start = time.perf_counter()
    for k, a in enumerate(arrivals):
        now = time.perf_counter() - t_start
        if a.t > now:
            time.sleep(a.t - now)
        # fold the results of arrivals up to k - lag, in arrival order
        need = k - lag + 1
        t_wait = time.perf_counter()
        while True:
            with lock:
                while folded < need and folded in done:
                    rec = done[folded]
                    if rec is not None:
                        prefix.append(rec)
                        # only well-sampled candidates can become the best fit
                        if rec["n"] >= min_best_packets and rec["chi2"] < best["chi2"]:
                            best.update(chi2=rec["chi2"], tau0=rec["tau0"], beta=rec["beta"],
                                        m0=rec["m0"], d_m=rec["d_m"])
                    folded += 1
                ready = folded >= need
            if ready or time.perf_counter() - t_wait > 30.0:
                break
            time.sleep(0.0002)
        have_best = math.isfinite(best["chi2"])
        b = dict(best)
        if k % 50 == 0 and have_best:
            sur = surrogate_estimate(prefix)
            if sur is not None:
                # move the proposal centre to the surrogate's vertex, keeping m0/d
                # on the line that gives its tau0 (tau0 is linear in m0/d)
                center = dict(b)
                center["beta"] = sur["beta"]
                center["m0"] = b["m0"] * sur["tau0"] / b["tau0"]
                surrogate_center.update(center)
        if surrogate_center:
            b = dict(b, **surrogate_center)
        if k < explore * len(arrivals) or not have_best:
            params = dict(beta=a.beta, m0=a.m0, d_m=a.d_m)
        else:
            scale = max(0.02, 0.3 * (1.0 - k / len(arrivals)))
            params = dict(beta=b["beta"] * math.exp(scale * rng.standard_normal()),
                          m0=b["m0"] * math.exp(scale * rng.standard_normal()),
                          d_m=b["d_m"] * math.exp(scale * rng.standard_normal()))
            params["beta"] = min(max(params["beta"], 1.0), 20.0)
        wl = W.cfg5_request(W.Arrival(t=a.t, n_packets=a.n_packets, seed=a.seed, **params),
                            **probe)
        cloud = pdv.Cloud(ctx, wl)
        clouds.append(cloud)
        req = pdv.Request(cloud, wl, raw=True, counters=False)
        t0 = time.perf_counter()
        while True:
            try:
                ticket = pdv.pdv_submit(ctx.handle, req.c)
                break
            except pdv.PdvError as e:
                if e.status != pdv.PDV_EAGAIN:
                    raise
                res.rejected += 1
                time.sleep(0.001)
        with lock:
            pending[ticket] = (req, cloud, t0, params, k, wl)
        res.submitted += 1
    done_submitting.set()
    th.join()
    res.wall_s = time.perf_counter() - t_start
    res.records = [done[k] for k in sorted(done) if done[k] is not None]
    res.kept.sort(key=lambda x: x[0])
    res.best = {"chi2": math.inf}
    for rec in res.records:
        if rec["n"] >= min_best_packets and rec["chi2"] < res.best["chi2"]:
            res.best = dict(rec)
    for c in clouds:
        c.close()
    return res


def summary(res: SweepResult, hidden: dict) -> dict:
    lat = np.asarray(res.latencies_ms)
    return {
        "requests": res.submitted, "completed": res.completed, "rejected_retries": res.rejected,
        "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
        "spectra_per_s": res.completed / res.wall_s if res.wall_s else None,
        "best_candidate": {k: res.best.get(k) for k in ("beta", "m0", "d_m", "tau0", "chi2")},
        "recovered": surrogate_estimate(res.records),
        "hidden": hidden,
    }
