#!/usr/bin/env python
"""Benchmark: alias-table build + sampling on GB300, one JSON line on rank 0.

Workload (default): one table of N = 1e8 FP32 weights w_i = 1/rank^1.0 with
the ranks randomly permuted (seed 3) -- the paper's shuffled power law --
built with PSA, then 1e9 samples drawn by Walker's rule (Philox seed 2).
A step is one build plus the samples.  Inputs (400 MB weights, 800 MB table,
4 GB samples) are larger than L2, so no L2 flush is needed between steps.

`value` is build throughput (items/s) from CUDA events around the build
kernels of every timed step; `samples_per_s` comes from the events around
the sampler.  Under torchrun every rank builds and samples its own table (an
independent problem, no data-path collective): scaling is weak and `value`
sums all ranks' items over the slowest rank's time.

`--impl reference` times the CPU oracle (Vose's FP64 construction) on the
host cores for the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "alias build items/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
BUILD_BYTES_PER_ITEM = 32      # read w twice, write + read lh, write rows
SAMPLE_BYTES_PER_DRAW = 36     # one 32-byte row sector + a 4-byte output
KERNELS_PER_BUILD = 10         # sum, count, qsum, scatter, segscan, split ends, split, split fine, pack, info
# DRAM bytes the hardware moved per unit (dram__bytes_read.sum +
# dram__bytes_write.sum) in ncu captures of these kernels: the build at
# N = 2^25 items (sum 4.1, count 4.0, scatter 10.6, split 0.9, pack 15.6) and
# the naive sampler drawing 2^25 samples from a 2^25-row table (87.6 B of row
# sectors read + 4 B written per draw); both workloads exceed L2 and the
# traffic grows with the units, so a launch's traffic is these times its
# units.  To be re-measured whenever one of these kernels changes.
BUILD_TRAFFIC_PER_ITEM = 35.2
SAMPLE_TRAFFIC_PER_DRAW = 91.5
KERNELS_PER_SAMPLE = 1
# batched build/sample are timed separately (extra keys), not in gpu_launches


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["wrs", "reference"], default="wrs")
    ap.add_argument("--n", type=int, default=100_000_000)
    ap.add_argument("--samples", type=int, default=1_000_000_000)
    ap.add_argument("--section", type=int, default=1024)
    ap.add_argument("--dist", default="zipf",
                    choices=["zipf", "zipf0.5", "uniform", "exponential", "gamma"],
                    help="weights of the single table (default: shuffled power law)")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the host-side mass check of the timed table")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-psa-plus", action="store_true",
                    help="skip the PSA+ build (Sec. 4) timed on the same table")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--build-only", action="store_true",
                    help="time the build alone (no sampling legs, batched or serving)")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="also measure the request loop's capacity and replay the stream "
                         "at 0.3, 0.6 and 0.9 of it (--serve-requests requests each)")
    ap.add_argument("--batch-tables", type=int, default=100_000)
    ap.add_argument("--sampler-heatmap", action="store_true",
                    help="also time every sampling mode over a grid of table sizes and draw "
                         "counts (Sec. 6, sampler comparison)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the split and pack steps for both split methods and "
                         "every section size on this table (Sec. 6, split/pack variants)")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    from paper_2106_12270_gb300 import replicas
    return replicas.env()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def oracle_build_items_per_s(w, reps_budget_s: float = 20.0):
    """Time the FP64 Vose oracle (single thread) on `w`; returns (items/s, runs)."""
    import oracle
    oracle.build()
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.vose(w)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > reps_budget_s or len(times) >= 3:
            break
    return w.size / statistics.median(times), len(times)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2106_12270_gb300 import inputs
    import oracle
    oracle.build()
    # bounded sample of the workload: the first 1e7 items of the same array
    # recipe keep each step near one second of single-core work
    n = min(args.n, 10_000_000)
    w = inputs.zipf_permuted(n, 3)
    for _ in range(args.warmup):
        oracle.vose(w)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.vose(w)
        ts.append(time.perf_counter() - t0)
    sec = sum(ts) / len(ts)
    value = n / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "items/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"single table, shuffled power law s=1.0 (seed 3), "
                               f"oracle sample N={n} of N={args.n}", "n": n},
        "cpu_baseline": {"value": value, "unit": "items/s", "cores": 1, "kind": "oracle",
                         "sample": f"Vose FP64 build of N={n} shuffled-power-law weights"},
        "e2e": {"value": value, "unit": "items/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import _build, inputs, replicas

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    wrs.lib()

    n, count = args.n, args.samples
    cfg = wrs.config(args.section)
    seed = replicas.rank_seed(args.seed if args.seed is not None else
                              {"zipf": 3, "zipf0.5": 5, "uniform": 1, "exponential": 4,
                               "gamma": 7}[args.dist],
                              rank)
    w_host = inputs.by_name(args.dist, n, seed)
    w = torch.from_numpy(w_host).cuda()
    builder = wrs.Builder(n, cfg)
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    if args.build_only:
        count = 0
        args.no_batched = args.no_serving = args.no_e2e = args.no_accuracy = True
    out = torch.empty(max(count, 1), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        wrs.build_rows(w, rows, builder.ws, builder.info, cfg)
        if evs:
            evs[1].record(stream)
        if not args.build_only:
            wrs.sample_rows(rows, n, 0, count, 2, out)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = wrs.parse_info(builder.info)
    if info["status"] != wrs.OK:
        raise RuntimeError(f"build failed: {info}")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)  # let the sampler see the region
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    build_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    sample_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    total_ms, build_ms, sample_ms = replicas.max_over_ranks([total_ms, build_ms, sample_ms],
                                                            dist, "cuda")
    ms_per_step = total_ms / args.steps

    # end to end through the C ABI with host buffers (wrs_build_rows_host):
    # pinned weights in, table rows and summary out, copies inside the timed
    # region.  Two workspaces on two streams: one step's copy out overlaps
    # the next step's copy in and build (as a pipeline of requests would).
    e2e = None
    if not args.no_e2e:
        nbuf = 2
        w_pin = torch.from_numpy(w_host).pin_memory()
        rows_pin = [torch.empty(n, dtype=torch.int64).pin_memory() for _ in range(nbuf)]
        info_pin = [torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8).pin_memory()
                    for _ in range(nbuf)]
        hws = [torch.empty(wrs.build_host_workspace_bytes(n, cfg), dtype=torch.uint8,
                           device="cuda") for _ in range(nbuf)]
        streams = [torch.cuda.Stream() for _ in range(nbuf)]

        def e2e_steps(k0, k1):
            for k in range(k0, k1):
                b = k % nbuf
                wrs.build_rows_host(w_pin, rows_pin[b], hws[b], info_pin[b], cfg, streams[b])

        e2e_steps(0, max(2, args.warmup))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for st in streams:
            st.wait_event(a)
        e2e_steps(0, args.steps)
        for st in streams:
            stream.wait_stream(st)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b) / args.steps
        bad = [wrs.parse_info(x)["status"] for x in info_pin if wrs.parse_info(x)["status"]]
        if bad:
            raise RuntimeError(f"host build failed: {bad}")
        if not torch.equal(rows_pin[(args.steps - 1) % nbuf], rows.cpu()):
            raise RuntimeError("host build differs from the device build")
        e2e_ms = replicas.max_over_ranks([e2e_ms], dist, "cuda")[0]
        e2e = {"value": replicas.job_rate(n, world, e2e_ms), "unit": "items/s",
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 8 * n + wrs.INFO_BYTES,
               "ms_per_step": e2e_ms, "api": "wrs_build_rows_host",
               "pipelining": f"{nbuf} workspaces on {nbuf} streams"}

    # accuracy of the timed table: the reconstructed mass of every item
    # against N w_i / W in FP64 (plain numpy on the host; the stated bound is
    # |mass_i - N w_i/W| <= 1e-5 max(1, N w_i/W))
    accuracy = None
    if not args.no_accuracy:
        import numpy as np
        raw = rows.cpu().numpy().view(np.uint32).reshape(-1, 2)
        prob = raw[:, 0].view(np.float32).astype(np.float64)
        mass = prob + np.bincount(raw[:, 1], weights=1.0 - prob, minlength=n)
        wd = w_host.astype(np.float64)
        expect = wd * (n / float(np.sum(wd)))
        err = np.abs(mass - expect) / np.maximum(1.0, expect)
        accuracy = {"max_mass_error": float(err.max()), "mean_mass_error": float(err.mean()),
                    "bound": 1e-5, "items_checked": n,
                    "prefix_arithmetic": "exact 128-bit fixed-point prefix sums; sweep "
                                         "compares them at 2^-15 units (2^-46 of a bucket)"}
        del raw, prob, mass, wd, expect, err

    # sectioned sampling (Sec. 5): same draw count, samples grouped by section
    sec = {}
    for mode, name, rows_per in () if args.build_only else ((wrs.SAMPLE_CACHED, "cached", 8192),
                                 (wrs.SAMPLE_LIMITED, "limited", 8192),
                                 (wrs.SAMPLE_SMEM, "smem", 4096)):
        nsec = wrs.sample_sections(n, rows_per)
        cnt_t = torch.empty(nsec, dtype=torch.int64, device="cuda")
        off_t = torch.empty(nsec, dtype=torch.int64, device="cuda")
        wrs.sample_sectioned_rows(rows, n, count, 2, mode, rows_per, cnt_t, off_t, out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            wrs.sample_sectioned_rows(rows, n, count, 2, mode, rows_per, cnt_t, off_t, out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        sec[name] = {"ms": ms, "samples_per_s": world * count / (ms / 1e3),
                     "section_rows": rows_per}

    # Philox-rate probe: the sectioned samplers' generator calls and 4-byte
    # stores alone (same draw count); their arithmetic roofline
    if sec:
        wrs.diag_philox(count, 7, out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            wrs.diag_philox(count, 7, out)
        b.record(stream)
        torch.cuda.synchronize()
        ph_ms = a.elapsed_time(b) / args.steps
        for v in sec.values():
            v["frac_of_philox_probe"] = ph_ms / v["ms"]
        sec["philox_probe"] = {"ms": ph_ms, "samples_per_s": world * count / (ph_ms / 1e3),
                               "bound": "alu",
                               "what": "the same Philox-4x32-10 calls and 4-byte stores, "
                                       "no rows (wrs_diag_philox)"}

    # random-gather probe: the naive sampler's access pattern alone (same
    # table size, same number of draws), best of the three load paths
    probe = {}
    for flavor in () if args.build_only else (0, 1, 2):
        wrs.diag_random_gather(rows, n, count, 7, flavor, out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wrs.diag_random_gather(rows, n, count, 7, flavor, out)
        b.record(stream)
        torch.cuda.synchronize()
        probe[flavor] = a.elapsed_time(b)
    probe_ms = min(probe.values()) if probe else float("nan")

    psa_plus = None if (args.no_psa_plus or args.build_only) else \
        run_psa_plus(args, w, w_host, n, cfg, build_ms)
    batched = None if args.no_batched else run_batched(args, world, rank)
    serving_res = None if args.no_serving else run_serving(args, rank)
    if args.serve_sweep and serving_res is not None:
        serving_res["load_sweep"] = run_serving_sweep(args, rank)
    heatmap = run_sampler_heatmap(args) if args.sampler_heatmap else None
    ablation = run_ablation(args, w, n) if args.ablation else None

    hbm, peak_kind = peaks()
    build_gbs = BUILD_BYTES_PER_ITEM * n / (build_ms / 1e3) / 1e9
    sample_gbs = (SAMPLE_BYTES_PER_DRAW * count / (sample_ms / 1e3) / 1e9) if count else 0.0
    build_roof = {"bound": "hbm", "achieved": build_gbs, "peak": hbm, "unit": "GB/s",
                  "frac": build_gbs / hbm, "traffic": BUILD_TRAFFIC_PER_ITEM * n,
                  "traffic_unit": "bytes per build (ncu, scaled from N=2^25)",
                  "kernel": "build (10 kernels)",
                  "peak_kind": peak_kind}
    probe_gbs = (SAMPLE_BYTES_PER_DRAW * count / (probe_ms / 1e3) / 1e9) if probe else float("nan")
    sample_roof = {"bound": "hbm", "achieved": sample_gbs, "peak": hbm, "unit": "GB/s",
                   "frac": sample_gbs / hbm,
                   "traffic": SAMPLE_TRAFFIC_PER_DRAW * count if count else None,
                   "traffic_unit": "bytes per launch (ncu, scaled from 2^25 draws)",
                   "kernel": "k_sample_naive",
                   "peak_kind": peak_kind,
                   "random_gather_probe": {"achieved": probe_gbs, "unit": "GB/s",
                                           "frac_of_probe": (sample_gbs / probe_gbs) if probe else None,
                                           "ms": {str(k): v for k, v in probe.items()}}}
    dominant = sample_roof if (count and sample_ms >= build_ms) else build_roof

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nb = min(n, 10_000_000)
        ips, runs = oracle_build_items_per_s(w_host[:nb].copy())
        cpu = {"value": ips, "unit": "items/s", "cores": 1, "kind": "oracle",
               "sample": f"Vose FP64 build of the first {nb} weights, median of {runs} runs"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": replicas.job_rate(n, world, build_ms), "unit": "items/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u128 fixed point (build), u32 (sampling)",
            "data": "synthetic",
            "config": {"workload": f"single table N={n}, {args.dist} weights (seed {seed}); "
                                   f"build + {count} naive Walker samples (Philox seed 2)",
                       "n": n, "samples": count, "section_size": args.section,
                       "dist": args.dist,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}"},
            "build_ms": build_ms, "sample_ms": sample_ms,
            "samples_per_s": (world * count / (sample_ms / 1e3)) if count else None,
            "sectioned_sampling": sec,
            "batched": batched,
            "psa_plus": psa_plus,
            "serving": serving_res,
            **({"sampler_heatmap": heatmap} if heatmap is not None else {}),
            **({"ablation": ablation} if ablation is not None else {}),
            "roofline": dominant, "build_roofline": build_roof, "sample_roofline": sample_roof,
            "cpu_baseline": cpu, "e2e": e2e, "accuracy": accuracy, "clocks": clk,
            "gpu_launches": args.steps * (KERNELS_PER_BUILD + KERNELS_PER_SAMPLE),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args, world, rank):
    """Batched uneven tables: sizes log-uniform in [16, 65536] (seed 6),
    Gamma(0.1, 1) weights, one batched build launch plus 1e3 samples per
    table; compared with building the same tables one launch sequence at a
    time (timed on the first tables and scaled to the whole batch)."""
    import numpy as np
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs

    ntab = args.batch_tables
    sizes = inputs.log_uniform_sizes(ntab, 6 + rank, 16, 65536)
    off_np = np.zeros(ntab + 1, np.int64)
    off_np[1:] = np.cumsum(sizes)
    total = int(off_np[-1])
    torch.cuda.manual_seed(7 + rank)
    w = torch._standard_gamma(torch.full((total,), 0.1, device="cuda")).float()
    off = torch.from_numpy(off_np).cuda()
    rows = torch.empty(total, dtype=torch.int64, device="cuda")
    order = torch.from_numpy(wrs.batch_order(off_np).astype(np.int32)).cuda()
    bb = wrs.BatchBuilder(total, ntab)
    per_table = 1000
    cnt_off = torch.arange(0, (ntab + 1) * per_table, per_table, dtype=torch.int64, device="cuda")
    out = torch.empty(ntab * per_table, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(st=None):
        bb.build(w, off, rows, order, stream=st)
        wrs.sample_batched_rows(rows, off, ntab, cnt_off, 2, out, stream=st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # segment-to-block tiling picked by the autotuner (times every candidate
    # on this batch; later builds use the fastest)
    best, cand = bb.autotune(w, off, rows, order, force=True)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    bms, sms = [], []
    for _ in range(args.steps):
        ev[0].record(stream)
        bb.build(w, off, rows, order)
        ev[1].record(stream)
        wrs.sample_batched_rows(rows, off, ntab, cnt_off, 2, out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        bms.append(ev[0].elapsed_time(ev[1]))
        sms.append(ev[1].elapsed_time(ev[2]))
    summ = bb.summaries()
    ok = int((summ["status"] == wrs.OK).sum())
    mass_err = _batched_mass_error(rows, w, off, ntab)
    build_ms = statistics.mean(bms)
    sample_ms = statistics.mean(sms)

    # the same step captured once as a CUDA graph and replayed
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step(torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    gms = []
    for _ in range(args.steps):
        ev[0].record(stream)
        g.replay()
        ev[1].record(stream)
        torch.cuda.synchronize()
        gms.append(ev[0].elapsed_time(ev[1]))
    graph_ms = statistics.mean(gms)

    # baseline: the plain single-table path, one launch sequence per table
    probe = min(ntab, 2000)
    b1 = wrs.Builder(65536)
    r1 = torch.empty(65536, dtype=torch.int64, device="cuda")
    for t in range(min(probe, 50)):
        b1.build(w[off_np[t]:off_np[t + 1]], r1[: sizes[t]])
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for t in range(probe):
        b1.build(w[off_np[t]:off_np[t + 1]], r1[: sizes[t]])
    b.record(stream)
    torch.cuda.synchronize()
    probe_ms = a.elapsed_time(b)
    frac = sizes[:probe].sum() / sizes.sum()
    per_table_ms = probe_ms / frac
    return {"tables": ntab, "items": total, "tables_ok": ok, "build_ms": build_ms,
            "items_per_s": total / (build_ms / 1e3),
            "build_gbs": 36 * total / (build_ms / 1e3) / 1e9,
            "per_table_launch_ms": per_table_ms,
            "per_table_probe": f"first {probe} tables timed, scaled by item share {frac:.4f}",
            "speedup_vs_per_table": per_table_ms / build_ms,
            "samples": ntab * per_table, "sample_ms": sample_ms,
            "samples_per_s": ntab * per_table / (sample_ms / 1e3),
            "tuning": {"best": best,
                       "candidates": [{k: c[k] for k in ("threads", "chunk", "ms")}
                                      for c in cand]},
            "graph_step_ms": graph_ms,
            "graph_items_per_s": total / (graph_ms / 1e3),
            "max_mass_error": mass_err, "mass_error_bound": 1e-5}


def _batched_mass_error(rows, w, off, ntab):
    """max over every item of every table of |mass_i - N_t w_i/W_t| /
    max(1, N_t w_i/W_t), in FP64 on the device (torch ops: a measurement of
    the built tables, not part of the build)."""
    import torch
    dev = rows.device
    sizes = off[1:] - off[:-1]
    tid = torch.repeat_interleave(torch.arange(ntab, device=dev), sizes)
    raw = rows.view(torch.int32).view(-1, 2)
    prob = raw[:, 0].contiguous().view(torch.float32).double()
    alias = raw[:, 1].long() + off[:-1][tid]
    mass = prob.clone()
    mass.index_add_(0, alias, 1.0 - prob)
    del alias
    wd = w.double()
    Wt = torch.zeros(ntab, dtype=torch.float64, device=dev).index_add_(0, tid, wd)
    Wi = Wt[tid]
    expect = wd * sizes[tid].double() / Wi.clamp(min=1e-300)
    err = (mass - expect).abs() / expect.clamp(min=1.0)
    err = torch.where(Wi > 0, err, torch.zeros_like(err))
    return float(err.max())


def _time_ms(fn, reps=3):
    """Mean device time of fn() over reps runs after one warm-up (CUDA events)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_sampler_heatmap(args):
    """Every sampling mode over table sizes x draw counts (the paper compares
    its samplers over both axes, Sec. 6): uniform weights, a fresh table per
    size.  Reports ms per cell and the fastest mode."""
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs

    sizes = [1 << k for k in (16, 20, 24, 27)]
    counts = [1 << k for k in (16, 20, 24, 28)]
    modes = [("naive", wrs.SAMPLE_NAIVE, 0), ("cached", wrs.SAMPLE_CACHED, 8192),
             ("limited", wrs.SAMPLE_LIMITED, 8192), ("smem", wrs.SAMPLE_SMEM, 4096),
             ("smem16k", wrs.SAMPLE_SMEM, 16384)]
    out = torch.empty(max(counts), dtype=torch.int32, device="cuda")
    cells = []
    for n in sizes:
        w = torch.from_numpy(inputs.uniform(n, 1)).cuda()
        b = wrs.Builder(n)
        rows = torch.empty(n, dtype=torch.int64, device="cuda")
        b.build(w, rows)
        torch.cuda.synchronize()
        for c in counts:
            cell = {"n": n, "count": c}
            for name, mode, sec_rows in modes:
                if mode == wrs.SAMPLE_NAIVE:
                    ms = _time_ms(lambda: wrs.sample_rows(rows, n, 0, c, 2, out[:c]))
                else:
                    nsec = wrs.sample_sections(n, sec_rows)
                    cnt = torch.empty(nsec, dtype=torch.int64, device="cuda")
                    off = torch.empty(nsec, dtype=torch.int64, device="cuda")
                    ms = _time_ms(lambda: wrs.sample_sectioned_rows(rows, n, c, 2, mode, sec_rows,
                                                                    cnt, off, out[:c]))
                cell[name] = ms
            cell["best"] = min((k for k, _, _ in modes), key=lambda k: cell[k])
            cell["auto"] = wrs.sample_auto_choice(n, c)
            cells.append(cell)
        del w, rows, b
        torch.cuda.empty_cache()
    return {"weights": "uniform [0,1) (seed 1)", "unit": "ms", "cells": cells}


def run_psa_plus(args, w, w_host, n, cfg, psa_build_ms):
    """PSA+ (Sec. 4 "PSA+") on the bench table: greedy packing per 512-item
    partition chunk, PSA on the rest.  Each call reads the rest's size back
    once (a host sync), which the events around it include."""
    import numpy as np
    import torch

    import paper_2106_12270_gb300 as wrs

    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    ws = torch.empty(wrs.build_plus_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        greedy = wrs.build_rows_plus(w, rows, ws, info, cfg, 1)
    torch.cuda.synchronize()
    st = wrs.parse_info(info)["status"]
    if st != wrs.OK:
        raise RuntimeError(f"PSA+ build failed: status {st}")
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wrs.build_rows_plus(w, rows, ws, info, cfg, 1)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    res = {"ms": ms, "items_per_s": n / (ms / 1e3), "min_items": 1, "tile": 512,
           "greedy_items": greedy, "greedy_fraction": greedy / n,
           "speedup_vs_psa": psa_build_ms / ms}
    if not args.no_accuracy:
        raw = rows.cpu().numpy().view(np.uint32).reshape(-1, 2)
        prob = raw[:, 0].view(np.float32).astype(np.float64)
        mass = prob + np.bincount(raw[:, 1], weights=1.0 - prob, minlength=n)
        wd = w_host.astype(np.float64)
        expect = wd * (n / float(np.sum(wd)))
        res["max_mass_error"] = float((np.abs(mass - expect) / np.maximum(1.0, expect)).max())
        del raw, prob, mass, wd, expect
    del rows, info, ws
    torch.cuda.empty_cache()
    return res


def run_ablation(args, w, n):
    """Split and pack steps for both split methods (Sec. 4.1: partial p-ary
    vs binary search) and every section size (Sec. 4.2) on the bench table."""
    import torch

    import paper_2106_12270_gb300 as wrs

    res = []
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    for method, mname in ((wrs.SPLIT_PARY, "pary"), (wrs.SPLIT_BINARY, "binary")):
        for sec in (256, 512, 1024, 2048, 4096, 8192):
            cfg = wrs.config(sec, method)
            ws = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
            wrs.step_total(w, ws, cfg)
            wrs.step_partition(w, ws, cfg)
            split_ms = _time_ms(lambda: wrs.step_split(n, ws, cfg))
            pack_ms = _time_ms(lambda: wrs.step_pack(n, rows, ws, cfg))
            res.append({"split": mname, "section": sec, "split_ms": split_ms, "pack_ms": pack_ms})
            del ws
            torch.cuda.empty_cache()
    # pack designs of Sec. 4.2 (Fig. 3) on the same split state; all write
    # the same rows
    cfg = wrs.config(args.section)
    ws = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    wrs.step_total(w, ws, cfg)
    wrs.step_partition(w, ws, cfg)
    wrs.step_split(n, ws, cfg)
    variants = []
    for v, name in ((0, "one thread per section, weights gathered by index"),
                    (1, "one thread per section, weights in the lists"),
                    (2, "one warp per section, staged in shared memory, one lane sweeps"),
                    (3, "merge path over the section (production pack)")):
        if v == 3:
            fn = lambda: wrs.step_pack(n, rows, ws, cfg)
        else:
            fn = lambda v=v: wrs.diag_pack_variant(w, n, rows, ws, cfg, v)
        variants.append({"variant": v, "design": name, "pack_ms": _time_ms(fn)})
    del ws
    torch.cuda.empty_cache()
    return {"n": n, "dist": args.dist, "steps": res, "section": args.section,
            "pack_variants": variants}


def run_serving(args, rank):
    """Request loop: a Poisson stream (seed 5) of builds (10%, log-uniform
    1e3..1e7 items, uniform or shuffled power law), sample requests (85%,
    log-uniform 1e2..1e6 draws against resident tables) and releases (5%),
    admitted under an 80 GB HBM budget; latency from submit to completion."""
    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs, serving

    ops = inputs.serving_stream(args.serve_requests, 5 + rank, args.serve_rate)
    srv = wrs.Server(80 << 30, 4)
    try:
        warm = inputs.serving_stream(200, 99, args.serve_rate, build_range=(1_000, 100_000))
        serving.replay(srv, warm)
        srv.close()
        srv = wrs.Server(80 << 30, 4)
        _, _, _, status = serving.replay(srv, ops)
        st = srv.stats()
    finally:
        srv.close()
    ok = sum(1 for v in status.values() if v == wrs.OK)
    wall = st["wall_s"]
    return {"requests": len(ops), "ok": ok, "arrival_rate_per_s": args.serve_rate,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "requests_per_s": st["completed"] / wall if wall else None,
            "items_built_per_s": st["items_built"] / wall if wall else None,
            "samples_per_s": st["samples_drawn"] / wall if wall else None,
            "steps": st["steps"], "mean_step_requests": st["mean_step_requests"],
            "peak_bytes": st["peak_bytes"], "budget_bytes": 80 << 30}


def run_serving_sweep(args, rank):
    """Capacity of the request loop (the whole stream submitted at once,
    completions per second), then the Poisson stream replayed in real time at
    0.3, 0.6 and 0.9 of that capacity: latency against load."""
    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs, serving

    def run(rate, realtime):
        ops = inputs.serving_stream(args.serve_requests, 5 + rank, rate)
        srv = wrs.Server(80 << 30, 4)
        try:
            _, _, _, status = serving.replay(srv, ops, realtime=realtime)
            st = srv.stats()
        finally:
            srv.close()
        wall = st["wall_s"]
        return {"requests": len(ops), "ok": sum(1 for v in status.values() if v == wrs.OK),
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                "requests_per_s": st["completed"] / wall if wall else None,
                "mean_step_requests": st["mean_step_requests"]}

    cap = run(1e9, False)   # every arrival at time ~0: the loop's own rate
    capacity = cap["requests_per_s"]
    points = []
    for f in (0.3, 0.6, 0.9):
        r = run(f * capacity, True)
        r["load"] = f
        r["arrival_rate_per_s"] = f * capacity
        points.append(r)
    return {"capacity_requests_per_s": capacity, "saturated": cap, "points": points}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
