#!/usr/bin/env python3
"""Benchmark of the level-synchronous planar Quickhull on GB300.

One step = one hull of 1e8 uniform-square points and one hull of 1e8
uniform-disk points (FP64, SoA, seeds 1 and 2), the paper's 1e8-point
single-hull pass (Sec. 5.2 sizes) on synthetic stand-ins for its datasets.
Inputs are resident in HBM before the timed region; each 1.6 GB input is
larger than L2, so no flush is needed between steps.

Reported (one JSON line on rank 0):
  value       Gpoints/s over the timed steps (device time, CUDA events);
  batched     the 4096-set workload (sizes log-uniform in [64, 1e6], mixed
              distributions) in one vq_hull2d_batched call vs 4096
              sequential vq_hull2d calls on the same device-resident sets:
              hulls/s of both, and whether every hull is identical;
  serving     Poisson arrivals of requests (sizes log-uniform in [100, 1e7],
              mixed distributions) through the continuous-batching server
              (40 GB budget) vs one vq_hull2d_host call per request in
              arrival order: p50/p99 latency from arrival and hulls/s at
              rates up to past the plain path's saturation;
  e2e         the same through vq_hull2d_host from pinned host memory,
              host->device copy and result read-back inside the timing;
  roofline    the partition kernel (k_k1): paper-model bytes (16 per point
              classified or kept, Sec. 5.2) over its summed CUDA-event time,
              against the measured HBM copy bandwidth;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload.
--impl reference times the CPU oracle itself (the reference arm).
With --gpus N (torchrun) every rank runs the same workload on its own GPU
(replicas; weak scaling) and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Gpoints/s & % HBM peak per hull; batched hulls/s, p50/p99 vs plain (bit-exact)"
UNIT = "Gpoints/s"
WORKLOAD = "single hulls: uniform square + uniform disk, 1e8 FP64 SoA points each (seeds 1, 2)"
FULL_N = 100_000_000
# DRAM bytes the sieve moves per input point, from ncu captures of one
# sieve launch on 2e7-point square and disk hulls (profiles/): the input is
# read once (16 B per point) and the kept points are written.  Traffic grows
# in proportion to the points, so a launch's traffic is this times n.
SIEVE_DRAM_BYTES_PER_POINT = 16.08
# DRAM bytes of every kernel of one hull per input point (ncu, all launches
# of one 2e7-point hull; profiles/), per distribution.
HULL_DRAM_BYTES_PER_POINT = {"square": 16.25, "disk": 16.43}


def bench_configs(vq, torch, stream, dev, survivors, peak, reps=5):
    """The workload list's single-hull configurations: square 1e6 (seed 1),
    square / disk 1e8 (seeds 1 / 2, the step's inputs) and circle / Kuzmin 1e8
    (seeds 3 / 4): median ms per hull over CUDA-event timed calls after a
    warm-up, Gpoints/s, and the implementation model's bytes per hull (16 B
    per point read by the sieve, 20 B per point it keeps, 20 B per point read
    or kept at every level) over that time."""
    out = {}
    cases = [("1 square 1e6", "square", 1_000_000, None), ("2a square 1e8", "square", FULL_N, dev[0]),
             ("2b disk 1e8", "disk", FULL_N, dev[1]), ("3a circle 1e8", "circle", FULL_N, None),
             ("3b kuzmin 1e8", "kuzmin", FULL_N, None)]
    for name, dist, n, d in cases:
        if d is None:
            x, y = synth.workload(dist, n, workers=WORKERS)
            d = (torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
            del x, y
        o = torch.empty(n, dtype=torch.int32, device="cuda")
        vq.vq_hull2d(d[0], d[1], o, stream=stream)  # warm-up: workspace, graph
        st = vq.vq_last_stats()
        r = reps if dist != "circle" else 2
        ts = []
        for _ in range(r):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = vq.vq_hull2d(d[0], d[1], o, stream=stream).shape[0]
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        med = statistics.median(ts)
        model = 16.0 * n + 20.0 * st["read"][0] + 20.0 * (sum(st["read"]) + sum(st["written"]))
        out[name] = {"ms_per_hull": med, "gpoints_per_s": n / (med / 1e3) / 1e9, "h": int(h),
                     "kept_by_sieve": int(st["read"][0]), "levels": int(st["levels"]),
                     "model_bytes": model, "model_GBps": model / (med / 1e3) / 1e9,
                     "model_frac": model / (med / 1e3) / 1e9 / peak, "samples": r}
        del o
    torch.cuda.empty_cache()
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=FULL_N, help="points per hull (default: the 1e8 workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=30_000_000,
                    help="points per workload for the CPU-oracle baseline")
    ap.add_argument("--ppt", type=int, default=0, help="tuning: points per lane of the partition kernel")
    ap.add_argument("--small-max", type=int, default=0, help="tuning: small-segment threshold")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default knobs (by default vq_autotune picks them on the square "
                         "workload before timing)")
    ap.add_argument("--energy-seconds", type=float, default=3.0,
                    help="seconds of back-to-back steps for the energy figure (0: off)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration hull times")
    ap.add_argument("--serving-requests", type=int, default=1000)
    ap.add_argument("--profile-one", default="", choices=[""] + list(synth.DISTRIBUTIONS),
                    help="profiling aid: run --profile-reps hulls of --n points of this distribution "
                         "(the workload's seed), print their counters and exit")
    ap.add_argument("--profile-reps", type=int, default=3)
    ap.add_argument("--host-loop", action="store_true",
                    help="profiling aid: levels launched from the host (profilers see every kernel)")
    return ap.parse_args()


SEEDS = {"square": 1, "disk": 2, "circle": 3, "kuzmin": 4}


def profile_one(args):
    """The same hull --profile-reps times on cuda:0 (for ncu: the kernels of
    exactly these hulls run, nothing else), then one line of counters."""
    import torch
    import paper_2510_09417_gb300 as vq
    vq.load()
    if args.host_loop:
        vq.vq_set_config(host_loop=1)
    x, y = synth.points(args.profile_one, args.n, SEEDS.get(args.profile_one, 1))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    del x, y
    vq.vq_profile_read(reset=True)
    h = None
    for _ in range(max(1, args.profile_reps)):
        h = vq.vq_hull2d(xd, yd)
    torch.cuda.synchronize()
    p = vq.vq_profile_read(reset=True)
    st = vq.vq_last_stats()
    print(json.dumps({"profile_one": args.profile_one, "n": args.n, "reps": args.profile_reps, "h": int(h.shape[0]),
                      "launches": p["launches"], "k1_points_read": p["k1_points_read"],
                      "level_reads": st["read"][:8]}))


WORKERS = max(1, min(16, os.cpu_count() or 1))


def cpu_batched_baseline(x, y, offs, max_points=40_000_000):
    """The oracle on the first sets of the batched workload (at most
    max_points points in all, at least one set): one oracle hull per set on a
    thread pool over all host cores (the oracle's C call releases the GIL).
    Returns the rate of that sample."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    sizes = offs[1:] - offs[:-1]
    k = max(1, int(np.searchsorted(np.cumsum(sizes), max_points, side="right")))
    pts = int(offs[k])
    cores = os.cpu_count() or 1

    def one(s):
        a, b = int(offs[s]), int(offs[s + 1])
        return oracle.hull(x[a:b], y[a:b]).shape[0]

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, range(k)))
    sec = time.perf_counter() - t0
    return {"hulls_per_s": k / sec, "gpoints_per_s": pts / sec / 1e9, "cores": cores, "kind": "oracle",
            "sample": f"the first {k} of the {len(offs) - 1} sets ({pts:,} points), one oracle hull per set "
                      f"on a pool of {cores} threads", "seconds": sec}


def bench_batched(vq, torch, stream, steps, cpu=True):
    """One vq_hull2d_batched call over the 4096-set workload against 4096
    sequential vq_hull2d calls on the same device-resident sets; with cpu,
    the oracle on a bounded sample of the sets over all host cores."""
    x, y, offs, dists = synth.batched_sets(workers=WORKERS)
    nsets, total = len(offs) - 1, int(offs[-1])
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    od = torch.from_numpy(offs).cuda()
    hi = torch.empty(total, dtype=torch.int32, device="cuda")
    ho = torch.empty(nsets + 1, dtype=torch.int64, device="cuda")
    vq.vq_hull2d_batched(xd, yd, od, hi, ho, stream=stream)  # warm-up: workspace, graph
    k = max(1, min(steps, 3))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        vq.vq_hull2d_batched(xd, yd, od, hi, ho, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batched = e0.elapsed_time(e1) / k
    # sequential plain calls, one per set
    out = torch.empty(int((offs[1:] - offs[:-1]).max()), dtype=torch.int32, device="cuda")
    for s in range(min(nsets, 64)):
        vq.vq_hull2d(xd[offs[s]:offs[s + 1]], yd[offs[s]:offs[s + 1]], out, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(nsets):
        vq.vq_hull2d(xd[offs[s]:offs[s + 1]], yd[offs[s]:offs[s + 1]], out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    # every set's batched hull against its plain hull (untimed)
    hof = ho.cpu().numpy()
    mismatched = 0
    neq = torch.zeros((), dtype=torch.int64, device="cuda")
    for s in range(nsets):
        h = vq.vq_hull2d(xd[offs[s]:offs[s + 1]], yd[offs[s]:offs[s + 1]], out, stream=stream)
        if h.shape[0] != hof[s + 1] - hof[s]:
            mismatched += 1
        else:
            neq += (hi[hof[s]:hof[s + 1]] != h).sum()
    mismatched += int(neq.item() > 0)
    del xd, yd, od, hi, ho, out
    torch.cuda.empty_cache()
    cpu_base = cpu_batched_baseline(x, y, offs) if cpu else None
    del x, y
    return {"workload": f"{nsets} sets, sizes log-uniform in [64, 1e6], distributions mixed (seed 5)",
            "sets": nsets, "points": total,
            "batched_ms": ms_batched, "batched_hulls_per_s": nsets / (ms_batched / 1e3),
            "batched_gpoints_per_s": total / (ms_batched / 1e3) / 1e9,
            "sequential_ms": ms_seq, "sequential_hulls_per_s": nsets / (ms_seq / 1e3),
            "speedup": ms_seq / ms_batched, "identical_to_plain_calls": mismatched == 0,
            "cpu_baseline": cpu_base,
            "timing": f"CUDA events; batched: mean of {k} calls after one warm-up; sequential: one pass "
                      "after 64 warm-up calls; inputs resident in HBM"}


def bench_serving(vq, torch, nreq, budget=40 << 30, lanes=3):
    """Continuous-batching server vs one vq_hull2d_host call per request, on
    the same Poisson arrivals, at rates up to past the plain path's
    saturation."""
    import threading
    reqs = synth.serving_requests(nreq, rate_per_s=1.0)  # arrival times at rate 1; scaled per rate
    pts = [synth.points(r["dist"], r["n"], r["seed"], workers=WORKERS) for r in reqs]
    cap = max(r["n"] for r in reqs)
    hbuf = np.empty(cap, dtype=np.int32)

    def plain(rate):
        """One blocking vq_hull2d_host call per request in arrival order;
        latency = completion - arrival.  rate None: all arrive at once."""
        lat, hulls = [], []
        t0 = time.perf_counter()
        for r, (x, y) in zip(reqs, pts):
            ta = t0 + (r["t"] / rate if rate else 0.0)
            d = ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            h = vq.vq_hull2d_host(x, y, hull_idx=hbuf)
            lat.append(time.perf_counter() - ta)
            if rate is None:
                hulls.append(h.copy())
        return lat, time.perf_counter() - t0, hulls

    def served(rate):
        """Requests submitted at their arrival times from one thread; results
        taken in completion order; latency = (submit start - arrival) +
        the server's submit-to-completion time."""
        lat = [0.0] * nreq
        offset = {}
        hulls = [None] * nreq
        with vq.Server(mem_budget_bytes=budget, max_inflight=256, lanes=lanes) as srv:
            t0 = time.perf_counter()

            def submitter():
                for i, (r, (x, y)) in enumerate(zip(reqs, pts)):
                    ta = t0 + (r["t"] / rate if rate else 0.0)
                    d = ta - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    ts = time.perf_counter()
                    t = srv.submit(x, y)
                    offset[t] = (i, ts - ta)

            th = threading.Thread(target=submitter)
            th.start()
            got = []
            for _ in range(nreq):
                res = srv.wait_any(cap, timeout_ms=600_000)
                if res is None:
                    raise RuntimeError("server: no result within 600 s")
                got.append(res)
            th.join()
            wall = time.perf_counter() - t0
            info = srv.info()
        for t, h, ms in got:
            i, off = offset[t]
            lat[i] = off + ms / 1e3
            hulls[i] = h
        return lat, wall, hulls, info

    def pct(v, q):
        return float(np.percentile(np.asarray(v) * 1e3, q))

    vq.vq_hull2d_host(*pts[0], hull_idx=hbuf)  # warm-up
    lat_p, wall_p, hulls_p = plain(None)
    lat_s, wall_s, hulls_s, info_s = served(None)
    identical = all(np.array_equal(a, b) for a, b in zip(hulls_p, hulls_s))
    sat_plain, sat_served = nreq / wall_p, nreq / wall_s
    sweep = []
    for f in (0.25, 0.5, 0.9, 1.2):
        rate = f * sat_plain
        lp, wp, _ = plain(rate)
        ls, ws_, _, inf = served(rate)
        sweep.append({"rate_per_s": rate, "fraction_of_plain_saturation": f,
                      "plain": {"p50_ms": pct(lp, 50), "p99_ms": pct(lp, 99), "hulls_per_s": nreq / wp},
                      "served": {"p50_ms": pct(ls, 50), "p99_ms": pct(ls, 99), "hulls_per_s": nreq / ws_,
                                 "admitted_while_busy": inf["admitted_while_busy"],
                                 "max_busy_lanes": inf["max_busy_lanes"], "batches": inf["batches"]}})
    return {"workload": f"{nreq} requests per rate, sizes log-uniform in [100, 1e7] FP64 points, distributions "
                        "mixed, Poisson arrivals (seed 6); the plain path copies each request from pageable host "
                        "memory, the server stages submitted points in its pinned area",
            "points": int(sum(r["n"] for r in reqs)), "budget_bytes": budget, "lanes": lanes,
            "saturated": {"plain_hulls_per_s": sat_plain, "served_hulls_per_s": sat_served,
                          "plain_p50_ms": pct(lat_p, 50), "plain_p99_ms": pct(lat_p, 99),
                          "served_p50_ms": pct(lat_s, 50), "served_p99_ms": pct(lat_s, 99),
                          "served_peak_bytes": info_s["peak_bytes"], "served_batches": info_s["batches"]},
            "sweep": sweep, "identical_to_plain_calls": identical}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    from paper_2510_09417_gb300.replicas import dist_env as env
    return env()


def cpu_oracle_rate(n_sample: int):
    """Oracle (sequential C, one core) on the first n_sample points of each
    workload; returns (Gpoints/s, seconds, sample text)."""
    import oracle
    oracle.build()
    total_pts = 0
    total_s = 0.0
    for dist in ("square", "disk"):
        x, y = synth.workload(dist, FULL_N) if n_sample >= FULL_N else synth.points(
            dist, n_sample, synth.WORKLOAD_SEEDS[(dist, FULL_N)])
        t0 = time.perf_counter()
        oracle.hull(x, y)
        total_s += time.perf_counter() - t0
        total_pts += x.shape[0]
    sample = (f"first {n_sample:,} points of each of the square and disk 1e8 workloads "
              f"(same seeds), one oracle hull each, 1 thread")
    return total_pts / total_s / 1e9, total_s, sample


class ClockSampler:
    """nvidia-smi clock, power and throttle samples during a measured region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
                 str(self.interval_ms)],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            lines = f.read().splitlines()
        os.unlink(self.path)
        return self.summarize(lines, self.gpu)

    @staticmethod
    def summarize(lines, gpu: int):
        """Median SM clock and power, the clock ceiling and the active
        throttle reasons of one GPU's csv lines; None without samples."""
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != gpu:
                    continue
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons), "power_w": statistics.median(pw) if pw else None}


def measure_energy(step, gpu: int, points_per_step: int, seconds: float = 3.0, idle_seconds: float = 1.0):
    """Energy per hull, as in the paper's energy study but from the GPU's
    own power readings (nvidia-smi, NVML) instead of RAPL: the median board
    power while the GPU idles for idle_seconds, then while the step runs back
    to back for `seconds`.  Returns the energy per step in total and above
    idle, and Gpoints per joule."""
    import torch
    torch.cuda.synchronize()
    idle = ClockSampler(gpu, 100)
    idle.start()
    time.sleep(idle_seconds)
    ri = idle.stop()
    load = ClockSampler(gpu, 100)
    load.start()
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        step()
        n += 1
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    rl = load.stop()
    if not ri or not rl or ri.get("power_w") is None or rl.get("power_w") is None:
        return {"unavailable": "no power samples from nvidia-smi"}
    per_step_s = sec / n
    j_total = rl["power_w"] * per_step_s
    j_above = (rl["power_w"] - ri["power_w"]) * per_step_s
    return {"idle_w": ri["power_w"], "load_w": rl["power_w"], "steps": n, "seconds": sec,
            "joules_per_step": j_total, "joules_per_step_above_idle": j_above,
            "gpoints_per_joule": points_per_step / j_total / 1e9 if j_total > 0 else None,
            "load_clocks": {k: rl[k] for k in ("sm_mhz", "sm_max_mhz", "samples", "reasons")},
            "source": "nvidia-smi power.draw every 100 ms; idle-subtracted figure uses the idle median"}


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle, timed on this host."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    m = min(args.n, 10_000_000)
    data = [synth.points(d, m, synth.WORKLOAD_SEEDS[(d, FULL_N)]) for d in ("square", "disk")]
    for _ in range(args.warmup):
        for x, y in data:
            oracle.hull(x, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for x, y in data:
            oracle.hull(x, y)
    sec = time.perf_counter() - t0
    pts = 2 * m * args.steps
    value = pts / sec / 1e9
    sample = f"first {m:,} points of each of the square and disk 1e8 workloads per step, 1 thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        # the same workload as the device arm; each step hulls a bounded
        # sample of it (see cpu_baseline.sample)
        "config": {"workload": WORKLOAD, "points_per_hull": args.n, "hulls_per_step": 2,
                   "l2": "no flush: each input (1.6 GB at 1e8 points) exceeds L2",
                   "parallelism": "replicas x1", "sample_points_per_hull": m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.profile_one:
        return profile_one(args)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_2510_09417_gb300 as vq

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vq.load()
    if args.ppt:
        vq.vq_set_config(points_per_thread=args.ppt)
    if args.small_max:
        vq.vq_set_config(small_max=args.small_max)
    n = args.n
    if n == FULL_N:
        data = [synth.workload(d, n, workers=WORKERS) for d in ("square", "disk")]
    else:
        data = [synth.points(d, n, synth.WORKLOAD_SEEDS[(d, FULL_N)], workers=WORKERS) for d in ("square", "disk")]
    dev = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in data]
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in dev]
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_autotune and not (args.ppt or args.small_max):
        cfg, tms = vq.vq_autotune(dev[0][0], dev[0][1], reps=2, stream=stream)
        tuned = {"autotuned_on": "square workload", "median_ms": tms}

    def step():
        hs = []
        for (xd, yd), o in zip(dev, outs):
            hs.append(vq.vq_hull2d(xd, yd, o, stream=stream).shape[0])
        return hs

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        hull_sizes = step()
    survivors = []  # points the sieve kept per hull (level 0 reads them)
    for (xd, yd), o in zip(dev, outs):
        vq.vq_hull2d(xd, yd, o, stream=stream)
        survivors.append(int(vq.vq_last_stats()["read"][0]))
    def timed(profile: bool):
        # K steps between a barrier and a synchronize on both sides, CUDA
        # events on the launching stream; with profile on, the library also
        # brackets every kernel with events (per-kernel device times)
        vq.vq_set_config(profile=1 if profile else 0)
        vq.vq_profile_read(reset=True)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            hs = step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        p = vq.vq_profile_read(reset=True)
        vq.vq_set_config(profile=0)
        return e0.elapsed_time(e1), p, hs

    # the value: the timed region without per-kernel events; clocks sampled
    # during it.  The roofline: the same K steps again, each kernel timed
    # with CUDA events (their records cost a few percent of the step).
    clocks = ClockSampler(local)
    clocks.start()
    ms, prof_plain, hull_sizes = timed(False)
    clk = clocks.stop()
    ms_prof, prof, _ = timed(True)
    prof["launches"] = prof_plain["launches"]
    from paper_2510_09417_gb300.replicas import job_rate, max_over_ranks
    ms_max = max_over_ranks(ms, device="cuda")
    pts_step = 2 * n * ws
    value = job_rate(2 * n * args.steps, ws, ms_max / 1e3) / 1e9

    # roofline of the dominant kernel, the sieve: 16 bytes read per point and
    # 20 written per point it keeps (the level-0 reads), over its event time
    peak, peak_kind = peaks()
    kept = sum(survivors) * args.steps
    sv_bytes = 16.0 * 2 * n * args.steps + 20.0 * kept
    sv_s = prof["k0_ms"] / 1e3
    sv_launches = 2 * args.steps
    achieved = sv_bytes / sv_s / 1e9 if sv_s > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": SIEVE_DRAM_BYTES_PER_POINT * n, "peak_kind": peak_kind,
                "kernel": "k_sieve (pre-filter + extreme pass: one streaming read of every point)",
                "bytes_per_launch": sv_bytes / sv_launches,
                "ms_per_launch": prof["k0_ms"] / sv_launches,
                "timing": "CUDA events around every sieve launch, over a second pass of the same K steps "
                          f"({ms_prof / args.steps:.3f} ms per step with the events, "
                          f"{ms / args.steps:.3f} ms without)"}
    # the recursion after the sieve: the level loop hands its segments to the
    # persistent worklist (at level 0 on these inputs), whose time is spent
    # on the recursion's dependent chain of tasks, not on bytes (under 0.2 B
    # per input point, profiles/bench_launch_list.md); the level-loop
    # partition kernel runs only above the handover level
    calls = max(prof["calls"], 1)
    roofline["other_kernels"] = {
        "k_wl (persistent worklist, the recursion below the handover level)": {
            "bound": "latency", "ms_per_hull": prof["k5_ms"] / calls,
            "points_classified_per_hull": prof["k1_points_read"] / calls},
        "k_k1w (level-loop partition, levels above the handover)": {
            "launches": int(prof["k1_launches"]), "ms_per_hull": prof["k1_ms"] / calls}}
    # the whole hull: DRAM bytes per hull (ncu, all kernels) over the device
    # time per hull of the value's timed region
    hull_ms = ms_max / args.steps / 2
    e2e_bytes = sum(HULL_DRAM_BYTES_PER_POINT[d] * n for d in ("square", "disk")) / 2
    roofline["e2e_frac"] = {
        "value": e2e_bytes / (hull_ms / 1e3) / 1e9 / peak, "dram_bytes_per_hull": e2e_bytes,
        "ms_per_hull": hull_ms,
        "how": "DRAM bytes of every kernel of one hull (ncu dram__bytes_read.sum + dram__bytes_write.sum at "
               "2e7 points, per point, scaled to the hull's points) over the device time per hull of the "
               "value's timed region, against the measured HBM peak"}

    # every configuration of the workload list: ms per hull (median of
    # CUDA-event timed calls), Gpoints/s and the implementation model's bytes
    configs = None
    if not args.no_configs and n == FULL_N:
        configs = bench_configs(vq, torch, stream, dev, survivors, peak)

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        pinned = [(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()) for x, y in data]
        hbuf = [np.empty(n, dtype=np.int32) for _ in pinned]

        def e2e_step():
            return [vq.vq_hull2d_host(px.numpy(), py.numpy(), hull_idx=hb).shape[0]
                    for (px, py), hb in zip(pinned, hbuf)]

        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 5))
        for _ in range(ksteps):
            hs = e2e_step()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        sec = max_over_ranks(sec, device="cuda")
        e2e = {"value": pts_step * ksteps / sec / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 16 * n, "d2h_bytes_per_step": 4 * int(sum(hs)),
               "steps": ksteps, "api": "vq_hull2d_host (pinned host buffers)"}

    # energy per hull (idle-subtracted board power over back-to-back steps)
    energy = None
    if ws == 1 and args.energy_seconds > 0:
        try:
            energy = measure_energy(step, local, 2 * n, seconds=args.energy_seconds)
        except Exception as exc:  # the figure is optional; the bench line is not
            energy = {"unavailable": f"{type(exc).__name__}: {exc}"}

    # batched and serving comparisons (one GPU: reported at N = 1)
    batched = serving = None
    if ws == 1 and not args.no_batched:
        batched = bench_batched(vq, torch, stream, args.steps, cpu=not args.no_cpu)
    if ws == 1 and not args.no_serving:
        serving = bench_serving(vq, torch, args.serving_requests)

    cpu = None
    if rank == 0 and not args.no_cpu and ws == 1:
        m = min(args.cpu_sample, n)
        rate, sec, sample = cpu_oracle_rate(m)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "seconds": sec}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_hull": n, "hulls_per_step": 2,
                       "l2": "no flush: each input (1.6 GB at 1e8 points) exceeds L2",
                       "parallelism": f"replicas x{ws}", "hull_sizes": hull_sizes},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "configs": configs,
            "batched": batched, "serving": serving, "energy": energy,
            "gpu_launches": int(prof["launches"]), "clocks": clk,
            "tuning": {"points_per_lane": int(vq.vq_get_config().points_per_thread),
                       "small_max": int(vq.vq_get_config().small_max),
                       "prefilter": int(vq.vq_get_config().prefilter),
                       "k1_shape": int(vq.vq_get_config().k1_shape), "autotune": tuned},
            "detail": {"profile": prof, "survivors_per_hull": survivors},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
