#!/usr/bin/env python
"""Benchmark: alias-table build + sampling on GB300, one JSON line on rank 0.

Workload (default): one table of N = 2^30 FP32 weights drawn from
Exponential(1) (seed 4), built with PSA (Sec. 2.2, Sec. 4), then 1e10
samples drawn by Walker's rule (Philox seed 2) in output chunks of at most
4e9 draws (one 16 GB buffer reused; the chunks are consecutive ranges of
one sample stream).  A step is one build plus the 1e10 draws.  Inputs
(4 GiB weights, 8 GiB table, 16 GB of samples per chunk) are larger than L2,
so no L2 flush is needed between steps.

`value` is build throughput (items/s) from CUDA events around the build
kernels of every timed step; `samples_per_s` comes from the events around
the sampler launches.  Under torchrun every rank builds and samples its own
table (an independent problem, no data-path collective): scaling is weak and
`value` sums all ranks' items over the slowest rank's time.

Extra keys (not in the timed step): the sectioned samplers on the same table
and draw count, the 1e8-item shuffled power law (build, 1e9 draws, mass
error), PSA+, the batched build of 100k uneven tables and the request loop.

`--impl reference` times the CPU oracle (Vose's FP64 construction) on the
host cores for the same metric, on a bounded sample of the same workload.
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
SECTOR_BYTES = 32
KERNELS_PER_BUILD = 10         # sum, count, qsum, scatter, segscan, split ends, split, split fine, pack, info
# DRAM bytes the hardware moved per unit (dram__bytes_read.sum +
# dram__bytes_write.sum) in ncu captures of these kernels, one kernel per capture: the build at
# N = 2^25 Exp(1) items (sum 4.09, count 4.08, scatter 10.72, split 1.04, pack 14.45) and
# the naive sampler drawing 2^25 samples from a 2^25-row table (87.6 B of row
# sectors read + 4 B written per draw); both workloads exceed L2 and the
# traffic grows with the units, so a launch's traffic is these times its
# units.  To be re-measured whenever one of these kernels changes.
BUILD_TRAFFIC_PER_ITEM = 34.39
SAMPLE_TRAFFIC_PER_DRAW = 91.5
SEEDS = {"zipf": 3, "zipf0.5": 5, "uniform": 1, "exponential": 4, "gamma": 7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["wrs", "reference"], default="wrs")
    ap.add_argument("--n", type=int, default=1 << 30)
    ap.add_argument("--samples", type=int, default=10_000_000_000)
    ap.add_argument("--chunk", type=int, default=4_000_000_000,
                    help="draws per sampling call (the output buffer holds one chunk)")
    ap.add_argument("--section", type=int, default=1024)
    ap.add_argument("--dist", default="exponential",
                    choices=["zipf", "zipf0.5", "uniform", "exponential", "gamma"],
                    help="weights of the single table (default: Exp(1), seed 4)")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the mass check of the timed table")
    ap.add_argument("--no-sectioned", action="store_true",
                    help="skip the sectioned samplers and the probes")
    ap.add_argument("--no-power-law", action="store_true",
                    help="skip the 1e8-item shuffled power-law table (extra key)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-psa-plus", action="store_true",
                    help="skip the PSA+ builds (Sec. 4)")
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
    """nvidia-smi clocks and throttle reasons, sampled during the timed region
    (read-only queries of the GPU this process runs on, named by its UUID:
    nvidia-smi numbers GPUs physically and ignores CUDA_VISIBLE_DEVICES)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def _gpu_id(self) -> str:
        try:
            import torch
            u = str(torch.cuda.get_device_properties(self.device).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            return str(self.device)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self._gpu_id(), f"--query-gpu={self.Q}",
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


def workload_seed(args) -> int:
    return args.seed if args.seed is not None else SEEDS[args.dist]


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


def oracle_sampler_rate(prob32, alias, draws_per_thread: int, threads: int):
    """The oracle's naive sampler (Walker, Philox seed 2) on an exported table,
    one contiguous range of the sample stream per host thread (the C call
    releases the GIL, so the threads run on separate cores).  Returns
    (samples/s, total draws)."""
    import concurrent.futures as cf

    import oracle
    oracle.build()
    oracle.sample_naive(prob32, alias, 0, 1024, 2)   # load the library

    def part(k):
        oracle.sample_naive(prob32, alias, k * draws_per_thread, draws_per_thread, 2)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(part, range(threads)))
    sec = time.perf_counter() - t0
    total = draws_per_thread * threads
    return total / sec, total


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2106_12270_gb300 import inputs
    import oracle
    oracle.build()
    # bounded sample of the workload: the first 1e7 items of the same array
    # recipe keep each step near a tenth of a second of single-core work
    seed = workload_seed(args)
    n = min(args.n, 10_000_000)
    w = inputs.by_name(args.dist, n, seed)
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
        "config": {"workload": f"single table, {args.dist} weights (seed {seed}), "
                               f"oracle sample N={n} of N={args.n}", "n": n},
        "cpu_baseline": {"value": value, "unit": "items/s", "cores": 1, "kind": "oracle",
                         "sample": f"Vose FP64 build of the first {n} of the N={args.n} "
                                   f"{args.dist} weights (seed {seed})"},
        "e2e": {"value": value, "unit": "items/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _events(k):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def _chunks(count: int, chunk: int):
    """(first, size) of the sampling calls covering draws 0..count-1."""
    out, first = [], 0
    while first < count:
        c = min(chunk, count - first)
        out.append((first, c))
        first += c
    return out


def device_mass_error(rows, w) -> float:
    """max_i |mass_i - N w_i/W| / max(1, N w_i/W) of a built table, in FP64 on
    the device with torch ops (a measurement of the result, not part of the
    build; W here is torch's FP64 sum of the weights)."""
    import torch
    n = w.numel()
    raw = rows.view(torch.int32).view(n, 2)
    prob = raw[:, 0].contiguous().view(torch.float32).double()
    mass = prob.clone()
    mass.index_add_(0, raw[:, 1].long(), 1.0 - prob)
    del prob
    wd = w.double()
    expect = wd * (n / float(wd.sum()))
    del wd
    err = float(((mass - expect).abs() / expect.clamp(min=1.0)).max())
    del mass, expect
    torch.cuda.empty_cache()
    return err


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
    if args.build_only:
        count = 0
        args.no_batched = args.no_serving = args.no_e2e = args.no_accuracy = True
        args.no_sectioned = args.no_power_law = True
    cfg = wrs.config(args.section)
    seed = replicas.rank_seed(workload_seed(args), rank)
    t_gen = time.perf_counter()
    w_host = inputs.by_name(args.dist, n, seed)
    gen_s = time.perf_counter() - t_gen
    w = torch.from_numpy(w_host).cuda()
    builder = wrs.Builder(n, cfg)
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    chunks = _chunks(count, args.chunk)
    out = torch.empty(max(min(count, args.chunk), 1), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        wrs.build_rows(w, rows, builder.ws, builder.info, cfg)
        if evs:
            evs[1].record(stream)
        for first, c in chunks:
            wrs.sample_rows(rows, n, first, c, 2, out[:c])
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
    evs = [_events(3) for _ in range(args.steps)]
    t_start, t_end = _events(2)
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
        e2e = run_e2e(args, w_host, rows, cfg, n, world, dist)

    # accuracy of the timed table: every item's reconstructed mass against
    # N w_i / W (the stated bound is |mass_i - N w_i/W| <= 1e-5 max(1, N w_i/W))
    accuracy = None
    if not args.no_accuracy:
        accuracy = {"max_mass_error": device_mass_error(rows, w), "bound": 1e-5,
                    "items_checked": n,
                    "prefix_arithmetic": "exact 128-bit fixed-point prefix sums; sweep "
                                         "compares them at 2^-15 units (2^-46 of a bucket)"}

    hbm, peak_kind = peaks()
    sampling = None if (args.no_sectioned or not count) else \
        run_sampling_extras(args, rows, n, count, out, world, sample_ms, hbm)

    power_law = None if args.no_power_law else run_power_law(args, world)
    psa_plus = None if (args.no_psa_plus or args.build_only) else \
        run_psa_plus(args, w, n, cfg, build_ms)
    batched = None if args.no_batched else run_batched(args, world, rank)
    serving_res = None if args.no_serving else run_serving(args, rank)
    if args.serve_sweep and serving_res is not None:
        serving_res["load_sweep"] = run_serving_sweep(args, rank)
    heatmap = run_sampler_heatmap(args) if args.sampler_heatmap else None
    ablation = run_ablation(args, w, n) if args.ablation else None

    build_gbs = BUILD_BYTES_PER_ITEM * n / (build_ms / 1e3) / 1e9
    sample_gbs = (SAMPLE_BYTES_PER_DRAW * count / (sample_ms / 1e3) / 1e9) if count else 0.0
    build_roof = {"bound": "hbm", "achieved": build_gbs, "peak": hbm, "unit": "GB/s",
                  "frac": build_gbs / hbm, "traffic": BUILD_TRAFFIC_PER_ITEM * n,
                  "traffic_unit": "bytes per build (ncu, scaled from N=2^25)",
                  "kernel": "build (10 kernels)", "algorithmic_bytes_per_item": 32,
                  "peak_kind": peak_kind}
    sample_roof = None
    if count:
        sectors_peak = hbm * 1e9 / SECTOR_BYTES
        sample_roof = {"bound": "hbm", "achieved": sample_gbs, "peak": hbm, "unit": "GB/s",
                       "frac": sample_gbs / hbm,
                       "traffic": SAMPLE_TRAFFIC_PER_DRAW * count / len(chunks),
                       "traffic_unit": "bytes per launch (ncu, scaled from 2^25 draws)",
                       "kernel": "k_sample_naive", "launches_per_step": len(chunks),
                       "algorithmic_bytes_per_draw": SAMPLE_BYTES_PER_DRAW,
                       "frac_of_sector_rate": (count / (sample_ms / 1e3)) / sectors_peak,
                       "sector_rate_peak": sectors_peak,
                       "peak_kind": peak_kind}
        if sampling and sampling.get("random_gather_probe"):
            pr = sampling["random_gather_probe"]
            sample_roof["random_gather_probe"] = pr
            sample_roof["frac_of_probe"] = (count / sample_ms) / (pr["count"] / pr["best_ms"])
    dominant = sample_roof if (count and sample_ms >= build_ms) else build_roof

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nb = min(n, 10_000_000)
        ips, runs = oracle_build_items_per_s(w_host[:nb].copy())
        cpu = {"value": ips, "unit": "items/s", "cores": 1, "kind": "oracle",
               "sample": f"Vose FP64 build of the first {nb} of the N={n} weights, "
                         f"median of {runs} runs"}
        if count:
            prob32, alias = wrs.rows_to_numpy(rows)
            threads = os.cpu_count() or 1
            per = max(1, min(count // threads, 20_000_000))
            rate, drawn = oracle_sampler_rate(prob32, alias, per, threads)
            cpu["sampler"] = {"value": rate, "unit": "samples/s", "cores": threads,
                              "kind": "oracle",
                              "sample": f"{drawn} draws (samples 0..{drawn - 1} of the timed "
                                        f"stream) from the GPU-built N={n} table, one range "
                                        f"per host thread"}
            del prob32, alias

    if rank == 0:
        line = {
            "metric": METRIC, "value": replicas.job_rate(n, world, build_ms), "unit": "items/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u128 fixed point (build), u32 (sampling)",
            "data": "synthetic",
            "config": {"workload": f"single table N={n}, {args.dist} weights (seed {seed}); "
                                   f"build + {count} naive Walker samples (Philox seed 2) "
                                   f"in {len(chunks)} calls of at most {args.chunk}",
                       "n": n, "samples": count, "chunk": args.chunk,
                       "section_size": args.section, "dist": args.dist,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}"},
            "build_ms": build_ms, "sample_ms": sample_ms,
            "samples_per_s": (world * count / (sample_ms / 1e3)) if count else None,
            "input_generation_s": gen_s,
            "sampling": sampling,
            "power_law_1e8": power_law,
            "batched": batched,
            "psa_plus": psa_plus,
            "serving": serving_res,
            **({"sampler_heatmap": heatmap} if heatmap is not None else {}),
            **({"ablation": ablation} if ablation is not None else {}),
            "roofline": dominant, "build_roofline": build_roof, "sample_roofline": sample_roof,
            "cpu_baseline": cpu, "e2e": e2e, "accuracy": accuracy, "clocks": clk,
            "gpu_launches": args.steps * (KERNELS_PER_BUILD + len(chunks)),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_e2e(args, w_host, rows, cfg, n, world, dist):
    """Build throughput through wrs_build_rows_host: pinned host weights in,
    host rows and summary out, every copy inside the timed region."""
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import replicas

    stream = torch.cuda.current_stream()
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
    a, b = _events(2)
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
    del hws, rows_pin, w_pin
    torch.cuda.empty_cache()
    return {"value": replicas.job_rate(n, world, e2e_ms), "unit": "items/s",
            "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 8 * n + wrs.INFO_BYTES,
            "ms_per_step": e2e_ms, "api": "wrs_build_rows_host",
            "pipelining": f"{nbuf} workspaces on {nbuf} streams"}


def run_sampling_extras(args, rows, n, count, out, world, naive_ms, hbm):
    """The sectioned samplers (Sec. 5) on the timed table with the same draw
    count and chunking, the mode AUTO picks, the Philox-rate probe (their
    arithmetic roofline) and the random-gather probe (the naive sampler's
    access pattern alone: the random-sector rate this GPU sustains)."""
    import torch

    import paper_2106_12270_gb300 as wrs

    stream = torch.cuda.current_stream()
    chunks = _chunks(count, args.chunk)
    res = {"naive": {"ms": naive_ms, "samples_per_s": world * count / (naive_ms / 1e3)}}
    for mode, name, rows_per in ((wrs.SAMPLE_CACHED, "cached", 8192),
                                 (wrs.SAMPLE_SMEM, "smem", 4096)):
        nsec = wrs.sample_sections(n, rows_per)
        cnt_t = torch.empty(nsec, dtype=torch.int64, device="cuda")
        off_t = torch.empty(nsec, dtype=torch.int64, device="cuda")

        def run():
            for k, (_, c) in enumerate(chunks):
                wrs.sample_sectioned_rows(rows, n, c, 2 + k, mode, rows_per, cnt_t, off_t, out[:c])

        run()
        torch.cuda.synchronize()
        a, b = _events(2)
        a.record(stream)
        for _ in range(args.steps):
            run()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        res[name] = {"ms": ms, "samples_per_s": world * count / (ms / 1e3),
                     "section_rows": rows_per, "speedup_vs_naive": naive_ms / ms,
                     "output_gbs": 4 * count / (ms / 1e3) / 1e9}
        del cnt_t, off_t
    res["auto_choice"] = wrs.sample_auto_choice(n, min(count, args.chunk))

    # Philox-rate probe: the sectioned samplers' generator calls and 4-byte
    # stores alone (same draw count)
    def philox():
        for k, (_, c) in enumerate(chunks):
            wrs.diag_philox(c, 7 + k, out[:c])

    philox()
    torch.cuda.synchronize()
    a, b = _events(2)
    a.record(stream)
    for _ in range(args.steps):
        philox()
    b.record(stream)
    torch.cuda.synchronize()
    ph_ms = a.elapsed_time(b) / args.steps
    for k in ("cached", "smem"):
        res[k]["frac_of_philox_probe"] = ph_ms / res[k]["ms"]
    res["philox_probe"] = {"ms": ph_ms, "samples_per_s": world * count / (ph_ms / 1e3),
                           "bound": "alu",
                           "what": "the same Philox-4x32-10 calls and 4-byte stores, "
                                   "no rows (wrs_diag_philox)"}

    # random-gather probe on the timed table: one chunk's draws, every load
    # path and a few launch shapes (CTAs per SM x loads in flight per thread);
    # the best is the random-sector rate this GPU sustains
    c0 = chunks[0][1]
    probe = {}
    for flavor, ctas, loads in ((0, 8, 8), (1, 8, 8), (2, 8, 8), (0, 16, 8), (0, 32, 16)):
        wrs.diag_random_gather(rows, n, c0, 7, flavor, out[:c0], ctas, loads)
        torch.cuda.synchronize()
        a, b = _events(2)
        a.record(stream)
        wrs.diag_random_gather(rows, n, c0, 7, flavor, out[:c0], ctas, loads)
        b.record(stream)
        torch.cuda.synchronize()
        probe[f"path{flavor}_ctas{ctas}_loads{loads}"] = a.elapsed_time(b)
    best = min(probe.values())
    res["random_gather_probe"] = {
        "count": c0, "ms": probe, "best_ms": best, "best": min(probe, key=probe.get),
        "gathers_per_s": c0 / (best / 1e3),
        "frac_of_sector_rate": (c0 / (best / 1e3)) / (hbm * 1e9 / SECTOR_BYTES),
        "what": "uniformly random 8-byte reads of the table and one 4-byte store each "
                "(wrs_diag_random_gather; path 0/1/2 = ld.global.nc/.cg/.cs)"}
    return res


def run_power_law(args, world):
    """The paper's shuffled power law at N = 1e8 (w = 1/rank, ranks permuted,
    seed 3): build, 1e9 naive draws (Philox seed 2), mass error of the table."""
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs

    n, count = 100_000_000, 1_000_000_000
    w = torch.from_numpy(inputs.zipf_permuted(n, 3)).cuda()
    cfg = wrs.config(args.section)
    b = wrs.Builder(n, cfg)
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        b.build(w, rows)
        wrs.sample_rows(rows, n, 0, count, 2, out)
    torch.cuda.synchronize()
    bm, sm = [], []
    for _ in range(args.steps):
        e = _events(3)
        e[0].record(stream)
        b.build(w, rows)
        e[1].record(stream)
        wrs.sample_rows(rows, n, 0, count, 2, out)
        e[2].record(stream)
        torch.cuda.synchronize()
        bm.append(e[0].elapsed_time(e[1]))
        sm.append(e[1].elapsed_time(e[2]))
    info = wrs.parse_info(b.info)
    hbm, _ = peaks()
    build_ms, sample_ms = statistics.mean(bm), statistics.mean(sm)
    # precision study: the split and pack steps with exact fixed point (the
    # build's), FP64 and paired-FP32 prefix arithmetic on the same lists
    precision = []
    ws2 = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    pws = torch.empty(wrs.diag_prec_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    rows2 = torch.empty(n, dtype=torch.int64, device="cuda")
    wrs.step_total(w, ws2, cfg)
    wrs.step_partition(w, ws2, cfg)
    for name, fn in (("exact fixed point (the build)",
                      lambda: (wrs.step_split(n, ws2, cfg), wrs.step_pack(n, rows2, ws2, cfg))),
                     ("FP64", lambda: wrs.diag_prec_split_pack(n, rows2, ws2, pws, cfg,
                                                               wrs.PREC_FP64)),
                     ("paired FP32 (compensated)",
                      lambda: wrs.diag_prec_split_pack(n, rows2, ws2, pws, cfg, wrs.PREC_FF))):
        ms = _time_ms(fn, max(3, args.steps))
        precision.append({"arithmetic": name, "split_pack_ms": ms,
                          "max_mass_error": device_mass_error(rows2, w)})
    del ws2, pws, rows2
    res = {"n": n, "samples": count, "weights": "w = 1/rank, ranks permuted (seed 3)",
           "status": info["status"], "nh": info["nh"],
           "build_ms": build_ms, "items_per_s": world * n / (build_ms / 1e3),
           "build_frac": BUILD_BYTES_PER_ITEM * n / (build_ms / 1e3) / 1e9 / hbm,
           "sample_ms": sample_ms, "samples_per_s": world * count / (sample_ms / 1e3),
           "max_mass_error": device_mass_error(rows, w), "mass_error_bound": 1e-5,
           "precision": precision}
    del w, b, rows, out
    torch.cuda.empty_cache()
    return res


def run_batched(args, world, rank):
    """Batched uneven tables: sizes log-uniform in [16, 65536] (seed 6),
    Gamma(0.1, 1) weights (seed 7, host-generated, the same arrays the
    oracle reads in the tests), one batched build launch plus 1e3 samples per
    table; compared with building every table of the batch with its own
    launch sequence of the single-table pipeline, from a C loop
    (wrs_diag_build_each)."""
    import numpy as np
    import torch

    import paper_2106_12270_gb300 as wrs
    from paper_2106_12270_gb300 import inputs

    ntab = args.batch_tables
    sizes = inputs.log_uniform_sizes(ntab, 6 + rank, 16, 65536)
    off_np = np.zeros(ntab + 1, np.int64)
    off_np[1:] = np.cumsum(sizes)
    total = int(off_np[-1])
    w = torch.from_numpy(inputs.gamma(total, 7 + rank, 0.1)).cuda()
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

    # baseline: the plain single-table pipeline, one launch sequence per
    # table for every table of the batch, issued by a C loop in the library
    each_ms, each_bad = wrs.diag_build_each(w, off_np, rows, 5)
    if each_bad:
        raise RuntimeError(f"per-table builds failed: {each_bad} tables")
    # the per-table rows equal the batched rows bit for bit (same arithmetic)
    each_rows = rows.clone()
    bb.build(w, off, rows, order)
    torch.cuda.synchronize()
    same = bool(torch.equal(each_rows, rows))
    del each_rows
    return {"tables": ntab, "items": total, "tables_ok": ok, "build_ms": build_ms,
            "items_per_s": total / (build_ms / 1e3),
            "build_gbs": 36 * total / (build_ms / 1e3) / 1e9,
            "per_table_launch_ms": each_ms,
            "per_table_baseline": "every table built by wrs_build_rows, one launch sequence "
                                  "per table from a C loop (wrs_diag_build_each), mean of "
                                  "5 passes over the batch",
            "per_table_rows_equal_batched": same,
            "speedup_vs_per_table": each_ms / build_ms,
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


def _psa_plus_once(args, w, n, cfg, psa_ms=None):
    """PSA+ (Sec. 4 "PSA+") on one table: greedy packing per tile of 1024
    items, PSA on the rest.  Each call reads the rest's size back
    once (a host sync), which the events around it include.  PSA is timed on
    the same table unless its time is given."""
    import numpy as np
    import torch

    import paper_2106_12270_gb300 as wrs

    stream = torch.cuda.current_stream()
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    if psa_ms is None:
        b = wrs.Builder(n, cfg)
        for _ in range(3):
            b.build(w, rows)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            a, e = _events(2)
            a.record(stream)
            b.build(w, rows)
            e.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(e))
        psa_ms = float(np.mean(ts))
        del b
    ws = torch.empty(wrs.build_plus_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        greedy = wrs.build_rows_plus(w, rows, ws, info, cfg, 1)
    torch.cuda.synchronize()
    st = wrs.parse_info(info)["status"]
    if st != wrs.OK:
        raise RuntimeError(f"PSA+ build failed: status {st}")
    ts = []
    for _ in range(args.steps):
        a, e = _events(2)
        a.record(stream)
        wrs.build_rows_plus(w, rows, ws, info, cfg, 1)
        e.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(e))
    ms = float(np.mean(ts))
    res = {"n": n, "ms": ms, "items_per_s": n / (ms / 1e3), "min_items": 1, "tile": 1024,
           "greedy_items": greedy, "greedy_fraction": greedy / n, "psa_ms": psa_ms,
           "speedup_vs_psa": psa_ms / ms}
    if not args.no_accuracy:
        res["max_mass_error"] = device_mass_error(rows, w)
    del rows, info, ws
    torch.cuda.empty_cache()
    return res


def run_psa_plus(args, w, n, cfg, psa_build_ms):
    """PSA+ on the timed table, and on uniform weights at the paper's sizes
    (Sec. 6.1 compares PSA+ with PSA on uniform weights)."""
    import torch

    from paper_2106_12270_gb300 import inputs

    res = {"main": _psa_plus_once(args, w, n, cfg, psa_build_ms)}
    for nu in (10_000_000, 100_000_000):
        wu = torch.from_numpy(inputs.uniform(nu, 1)).cuda()
        res[f"uniform_{nu}"] = _psa_plus_once(args, wu, nu, cfg)
        del wu
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
