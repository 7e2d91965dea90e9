#!/usr/bin/env python3
"""Benchmark: Count Sketch key updates/s (k=4, p=2^61-1) on GB300.

Default workload (one JSON line): the large single sketch -- 2^28 keys drawn
Zipf(1.1) over a universe of 2^32 mapped to 61-bit keys, unit weights, t=7
rows, m=2^16 counters per row (3.5 MiB of int64 counters), two-for-one
hashing.  One step = zero the counters, cs_update over the whole stream,
cs_estimate_f2 (every step of the path, in the library's kernels).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|large-twopoly|plain|plain-2^28|sweep|batched|query|...]

`value` is whole-job keys/s with the keys already resident in HBM (2 GiB per
rank, far larger than the 129 MB L2, so no flush is needed between steps).
`e2e` is the same metric through the C ABI from pinned host buffers: each step
calls cs_update_host (the library copies the keys host->device in chunks,
overlapped with the updates), estimates F2 and reads the 16-byte estimate
back.  `roofline` is for the dominant kernel (k_cs_update), timed by
CUDA events on its own stream.  `cpu_baseline` (rank 0, N=1) times the CPU
oracle on a bounded sample of the same stream on this host's cores.
--impl reference times the CPU oracle alone (this method has no other
reference implementation).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

P61 = (1 << 61) - 1

# Workloads other than the single-sketch ones print their own lines (bench_extra.py).
WORKLOADS = {
    # name: (n, t, m, mode, keys, weights)
    "large": dict(n=1 << 28, t=7, m=1 << 16, mode=0, keys="zipf", weights=None,
                  desc="large single sketch: 2^28 Zipf(1.1) keys over 2^32, unit weights, "
                       "t=7, m=2^16, two-for-one"),
    "large-twopoly": dict(n=1 << 28, t=7, m=1 << 16, mode=1, keys="zipf", weights=None,
                          desc="large single sketch, two polynomials per row"),
    "plain": dict(n=1 << 20, t=5, m=1024, mode=0, keys="uniform", weights="pm100",
                  desc="plain single sketch: 2^20 uniform keys < 2^61-1, int32 weights in "
                       "[-100,100], t=5, m=1024"),
    "plain-2^28": dict(n=1 << 28, t=5, m=1024, mode=0, keys="uniform", weights="pm100",
                       desc="plain sketch distribution at 2^28 keys"),
    "plain-anyr": dict(n=1 << 28, t=5, m=1000, mode=2, keys="uniform", weights="pm100",
                       desc="plain sketch distribution at 2^28 keys, m = 1000 buckets "
                            "(any-m map of Algorithm Mersenne-arb-r)"),
}

# DRAM bytes per key of k_cs_update (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of the workload's first 2^25 keys in the bench's launch
# configuration; the stream's traffic grows in proportion, so a launch's traffic
# is this times its keys.  Only workloads whose current kernel was captured.
MEASURED_TRAFFIC_PER_KEY = {
    "large": (308.491264e6 + 3.525888e6) / 2 ** 25,
    "plain-2^28": (402.739200e6 + 3.022336e6) / 2 ** 25,
}

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS) + sorted(EXTRA))
    ap.add_argument("--sketches", type=int, default=4096, help="batched workload: sketch count")
    ap.add_argument("--seed", type=int, default=2008)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the plain-2^28 and batched sub-results")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--keys", type=int, default=0,
                    help="override the workload's keys per step (small cases for profiling)")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload: use the library's default tuning instead of tuning")
    return ap.parse_args()


# ------------------------------------------------------------------ inputs

def make_inputs(wl: dict, seed: int, rank: int, n: int | None = None):
    n = wl["n"] if n is None else n
    s = seed + 1000003 * rank
    if wl["keys"] == "zipf":
        keys = datagen.zipf(s, 1.1, 1 << 32, n)
    else:
        keys = datagen.u64_below(s, P61, n)
    w = datagen.i32_range(s, -100, 100, n) if wl["weights"] == "pm100" else None
    return keys, w


def inputs_desc(wl: dict) -> str:
    k = ("Zipf(1.1) ranks over [1,2^32] by rejection-inversion, rank r -> key "
         "r*0x9E3779B97F4A7C15 mod 2^61" if wl["keys"] == "zipf"
         else "uniform below 2^61-1 (SplitMix64 words scaled by p)")
    w = "unit weights" if wl["weights"] is None else "int32 weights uniform in [-100,100]"
    return "%s; %s; seeded counter-based generator (datagen)" % (k, w)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            self.path = "/tmp/ms_bench_clocks_%d.csv" % os.getpid()
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + CLOCK_QUERY, "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------------ roofline

def mad_wide_per_entry(t: int, nf: int) -> int:
    """32x32->64 multiply-adds (mad.wide) one hashed entry costs in the 2^61-1,
    k = 4 update kernels, counted from the row code (ms_field.cuh, row_sd and
    powers3): per row 9 products (Karatsuba on signed 31-bit digits) and 1
    fold step (the low 30 bits of the last sum times 2^31, a wide
    multiply-add); per key x^2 (3) and x^3 (4)."""
    return 10 * t * nf + 7


def hbm_peak_gbs() -> tuple:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), \
            "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6787.9, "fallback: the pool's measured copy bandwidth recorded for this project"


def probe_peaks(ms) -> dict:
    """Integer-multiply peaks of this GPU, measured in this run: 64x64->128
    products (the roofline's denominator) and 32x32->64 multiply-adds (the
    instruction the kernels issue: the best of the dependent-chain and the
    16-chain probes)."""
    mul_rate, _ = ms.probe_mul128(variant=0, iters=1 << 12)
    madw_dep, _ = ms.probe_mul128(variant=1, iters=1 << 13)
    madw_ind, _ = ms.probe_mul128(variant=4, iters=1 << 12)
    return {"mul128_per_s": mul_rate, "mad_wide_dependent_per_s": madw_dep,
            "mad_wide_independent_per_s": madw_ind, "mad_wide_per_s": max(madw_dep, madw_ind)}


def roofline_8d(n: int, t: int, nf: int, bytes_per_key: int, kern_s: float, peaks: dict,
                hbm_gbs: float, hbm_src: str) -> dict:
    """The roofline of the hot-path table's measurement row:
        roofline_time = max(n * bytes_per_key / HBM, n * t (k-1) / PEAK_mul128)
    over all n keys of the launch (the method's work, whatever the kernel
    skips), frac = roofline_time / kernel time."""
    mul_per_key = t * 3 * nf
    hbm_s = n * bytes_per_key / (hbm_gbs * 1e9)
    mul_s = n * mul_per_key / peaks["mul128_per_s"]
    if mul_s >= hbm_s:
        r = {"bound": "alu", "achieved": n * mul_per_key / kern_s / 1e9,
             "peak": peaks["mul128_per_s"] / 1e9, "unit": "Gmul128/s"}
    else:
        r = {"bound": "hbm", "achieved": n * bytes_per_key / kern_s / 1e9, "peak": hbm_gbs,
             "unit": "GB/s"}
    r["frac"] = max(hbm_s, mul_s) / kern_s
    r.update({
        "formula": "max(n*bytes_per_key/HBM, n*t*(k-1)*polys/PEAK_mul128) / kernel time, "
                   "n = every key of the launch",
        "roofline_ms": max(hbm_s, mul_s) * 1e3, "hbm_leg_ms": hbm_s * 1e3, "mul_leg_ms": mul_s * 1e3,
        "kernel_ms": kern_s * 1e3, "mul128_per_key": mul_per_key, "bytes_per_key": bytes_per_key,
        "peak_source": "ms_probe_mul128 variant 0 (independent 64x64->128 products, low half by "
                       "multiplication, high half by __umul64hi, every SM), measured in this run; "
                       "HBM: " + hbm_src,
        "hbm": {"achieved_gbs": n * bytes_per_key / kern_s / 1e9, "peak_gbs": hbm_gbs,
                "frac": n * bytes_per_key / kern_s / 1e9 / hbm_gbs},
    })
    return r


def imad_fraction(entries: int, t: int, nf: int, kern_s: float, peaks: dict) -> dict:
    """Counted mad.wide per hashed entry at the measured 32x32->64 multiply-add rate."""
    per = mad_wide_per_entry(t, nf)
    rate = entries * per / kern_s
    return {"mad_wide_per_entry": per, "entries_per_launch": entries,
            "achieved_per_s": rate, "peak_per_s": peaks["mad_wide_per_s"],
            "frac": rate / peaks["mad_wide_per_s"],
            "peak_source": "ms_probe_mul128 variants 1 and 4 (mad.wide.u32: 8 dependent chains, "
                           "and 16 cross-coupled chains per thread), the larger, measured in this "
                           "run"}


# ------------------------------------------------------------------ cpu baseline

def cpu_baseline(wl: dict, seed: int, target_s: float, gpu_check=None) -> dict:
    """The CPU oracle on a bounded sample of the same stream, all host cores."""
    import oracle
    cores = os.cpu_count() or 1
    coeffs = oracle.sketch_coeffs(61, 1, 4, wl["t"], wl["mode"], seed)
    n_cal = 1 << 16
    keys, w = make_inputs(wl, seed, 0, n_cal)
    t0 = time.perf_counter()
    oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, keys, w, nthreads=cores)
    rate = n_cal / max(time.perf_counter() - t0, 1e-6)
    n = int(min(wl["n"], max(1 << 16, rate * target_s)))
    n = 1 << int(math.log2(n))
    keys, w = make_inputs(wl, seed, 0, n)
    t0 = time.perf_counter()
    C = oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, keys, w, nthreads=cores)
    f2 = oracle.f2_estimate(C)
    dt = time.perf_counter() - t0
    out = {"value": n / dt, "unit": "keys/s", "cores": cores, "kind": "oracle",
           "sample": "first %d keys of the same seeded stream (%.1f s of CPU time on %d threads)"
                     % (n, dt, cores)}
    if gpu_check is not None:
        out["parity_on_sample"] = bool(gpu_check(keys, w, C, f2))
    return out


# ------------------------------------------------------------------ our arm

def time_steps(ms, sk, keys, w, f2_out, steps: int, warmup: int, gpu_index: int, stream,
               barrier=None) -> dict:
    """Device time of `steps` steps (zero, update, F2) after `warmup`, with CUDA
    events on the launching stream around every update kernel, and the SM
    clocks sampled during the timed region.  Inputs smaller than twice the L2
    get a 512 MiB write before every timed step; only the steps are timed, and
    a step is one CUDA-graph replay (three short kernels, which eager launches
    would leave host-bound)."""
    import torch
    n = keys.numel() if keys.dtype != torch.int32 else keys.numel()
    bytes_per_key = 8 + (4 if w is not None else 0)
    dev = keys.device
    l2_bytes = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 129 << 20)
    small = n * bytes_per_key < 2 * l2_bytes

    def step():
        sk.reset()
        sk.update(keys, w)
        sk.estimate_f2(out=f2_out)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev) if small else None
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(steps):
        if small:
            flush.fill_(i & 255)
        sk.reset()
        ev[i][0].record(stream)
        sk.update(keys, w)
        ev[i][1].record(stream)
        sk.estimate_f2(out=f2_out)
    t_end.record(stream)
    torch.cuda.synchronize()
    ms_total = t_start.elapsed_time(t_end)
    kern_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
    if small:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        for _ in range(max(3, warmup)):
            graph.replay()
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 255)
            sev[i][0].record(stream)
            graph.replay()
            sev[i][1].record(stream)
        torch.cuda.synchronize()
        ms_total = sum(sev[i][0].elapsed_time(sev[i][1]) for i in range(steps))
    if barrier:
        barrier()
    clk = clocks.stop()
    del flush
    return {"ms_total": ms_total, "kern_ms": kern_ms, "small": small, "clocks": clk,
            "bytes_per_key": bytes_per_key}


def hashed_entries(sk, keys, w) -> int:
    """Entries one launch hashes (keys with a non-zero weight, or with the
    de-duplication table the distinct (block, key) entries): one untimed update
    with the library's statistics hook on."""
    import torch
    hashed_t = torch.zeros(1, dtype=torch.int64, device=keys.device)
    sk.set_stats(hashed_t)
    sk.reset()
    sk.update(keys, w)
    torch.cuda.synchronize()
    sk.set_stats(None)
    return int(hashed_t.item())


def plain_result(args, ms, peaks, hbm_gbs, hbm_src, workload: str = "plain-2^28") -> dict:
    """The plain distribution (uniform keys below p, weights in [-100, 100], t=5,
    m=1024) at 2^28 keys, where the hot-path target is judged (or, with
    workload="plain", at its specified 2^20 keys, L2 flushed before each step)."""
    import torch
    wl = WORKLOADS[workload]
    n, t, m = wl["n"], wl["t"], wl["m"]
    keys_np, w_np = make_inputs(wl, args.seed, 0)
    keys = torch.from_numpy(keys_np.view(np.int64)).cuda()
    w = torch.from_numpy(w_np).cuda()
    del keys_np, w_np
    sk = ms.Sketch(t=t, m=m, k=4, b=61, c=1, seed=args.seed, mode=0)
    f2_out = torch.empty(2, dtype=torch.int64, device="cuda")
    steps = max(10, min(args.steps, 60)) if n > (1 << 24) else max(50, min(args.steps, 200))
    r = time_steps(ms, sk, keys, w, f2_out, steps, args.warmup, 0,
                   torch.cuda.current_stream())
    kern_s = statistics.mean(r["kern_ms"]) * 1e-3
    roof = roofline_8d(n, t, 1, 12, kern_s, peaks, hbm_gbs, hbm_src)
    roof["imad"] = imad_fraction(n, t, 1, kern_s, peaks)
    roof["traffic"] = MEASURED_TRAFFIC_PER_KEY.get(workload, 0) * n or None
    size = "2^28 keys" if n == 1 << 28 else "2^20 keys, L2 flushed before each step"
    out = {"workload": wl["desc"] + " (%s, t=5, m=1024, weights in [-100,100])" % size,
           "value": n * steps / (r["ms_total"] * 1e-3), "unit": "keys/s",
           "ms_per_step": r["ms_total"] / steps, "steps": steps, "roofline": roof,
           "launch": sk.last_launch(), "f2_estimate": str(ms.u128_to_int(f2_out.cpu()))}
    if r["clocks"]:
        out["clocks"] = r["clocks"]
    del keys, w, sk
    torch.cuda.empty_cache()
    return out


def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    import paper_2008_08654_gb300 as ms

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    n, t, m, mode = wl["n"], wl["t"], wl["m"], wl["mode"]
    nf = 2 if mode == 1 else 1
    keys_np, w_np = make_inputs(wl, args.seed, rank)
    keys = torch.from_numpy(keys_np.view(np.int64)).to(dev)
    w = None if w_np is None else torch.from_numpy(w_np).to(dev)
    sk = ms.Sketch(t=t, m=m, k=4, b=61, c=1, seed=args.seed, mode=mode)
    f2_out = torch.empty(2, dtype=torch.int64, device=dev)

    barrier = dist.barrier if world > 1 else None
    r = time_steps(ms, sk, keys, w, f2_out, args.steps, args.warmup, local, stream, barrier)
    launch = sk.last_launch()
    ms_total, kern_ms, small, clk = r["ms_total"], r["kern_ms"], r["small"], r["clocks"]
    bytes_per_key = r["bytes_per_key"]
    if world > 1:
        tt = torch.tensor([ms_total], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
    f2_est = ms.u128_to_int(f2_out.cpu())

    # e2e through the C ABI from pinned host buffers (copies in the timed region)
    keys_h = torch.from_numpy(keys_np.view(np.int64)).pin_memory()
    w_h = None if w_np is None else torch.from_numpy(w_np).pin_memory()
    f2_h = torch.empty(2, dtype=torch.int64).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))

    def e2e_step():
        # cs_update_host: the library streams the host arrays in, copy and
        # update overlapped chunk by chunk
        sk.reset()
        sk.update_host(keys_h, w_h)
        sk.estimate_f2(out=f2_out)
        f2_h.copy_(f2_out, non_blocking=True)
        stream.synchronize()

    for _ in range(2):
        e2e_step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    assert ms.u128_to_int(f2_h) == f2_est
    del keys_h, w_h

    peaks = probe_peaks(ms)
    hashed = hashed_entries(sk, keys, w)
    global_counters = launch.get("place") in (2, 3)
    red_rate = None
    if global_counters:
        # scattered int32 atomic additions into an L2-resident buffer the size
        # of the replicas (the counter updates' own bound)
        words = 1 << max(5, ((max(1, launch.get("replicas") or 1) * t * m) - 1).bit_length())
        red_rate, _ = ms.probe_red(words=words, iters=512)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None

    value = world * n * args.steps / (ms_total * 1e-3)
    kern_avg_s = statistics.mean(kern_ms) * 1e-3
    hbm_gbs, hbm_src = hbm_peak_gbs()
    roofline = roofline_8d(n, t, nf, bytes_per_key, kern_avg_s, peaks, hbm_gbs, hbm_src)
    roofline["imad"] = imad_fraction(hashed, t, nf, kern_avg_s, peaks)
    roofline["imad"]["note"] = ("entries = what the launch hashed (with the de-duplication table, "
                                "the distinct (block, key) entries with their counts)")
    if global_counters:
        adds = hashed * t / kern_avg_s  # counter additions (one per row per hashed entry)
        roofline["l2_atomic"] = {
            "achieved": adds / 1e9, "peak": red_rate / 1e9, "unit": "Gadd/s",
            "frac": adds / red_rate,
            "peak_source": "ms_probe_red: scattered red.global.add.s32 into an L2-resident "
                           "buffer the size of the replicas, every SM, measured in this run"}
    roofline.update({
        "traffic": (MEASURED_TRAFFIC_PER_KEY[args.workload] * n
                    if args.workload in MEASURED_TRAFFIC_PER_KEY else None),
        "traffic_unit": "bytes per launch (ncu DRAM bytes of a 2^25-key capture, scaled)",
        "algorithmic_bytes": n * bytes_per_key,
        "kernel": "k_cs_update",
        "keys_per_launch": n,
        "hashed_entries_per_launch": hashed,
        "probes": peaks,
    })
    line = {
        "metric": "Count Sketch key updates/s (k=4, p=2^61-1)",
        "value": value,
        "unit": "keys/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": ms_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "keys_per_step_per_gpu": n, "t": t, "m": m, "k": 4,
                   "p": "2^61-1", "mode": "two-poly" if mode == 1 else "two-for-one",
                   "inputs": inputs_desc(wl), "seed": args.seed,
                   "l2": ("inputs (%d MiB per GPU) fit the L2: a 512 MiB write flushes it "
                          "before every timed step, and only the steps are timed; a step is one "
                          "CUDA-graph replay of zero + update + F2" % (n * bytes_per_key >> 20))
                         if small else
                         ("inputs (%d MiB per GPU) exceed the 129 MB L2; no flush" %
                          (n * bytes_per_key >> 20)),
                   "launch": launch, "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "e2e": {"value": world * n * e2e_steps / e2e_s, "unit": "keys/s",
                "h2d_bytes_per_step": n * bytes_per_key, "d2h_bytes_per_step": 16},
        # zero, update, (second-level table drain,) (replica reduce,) F2 per
        # timed step; the library drains its second-level key table after
        # de-duplicating updates (unit weights, global placement) of 2^22 keys
        # or more
        "gpu_launches": (3 + (1 if launch.get("replicas") else 0)
                         + (1 if (w is None and launch.get("place") == 2 and launch.get("replicas")
                                  and n >= 1 << 22) else 0)) * args.steps,
        "f2_estimate": str(f2_est),
    }
    if clk:
        line["clocks"] = clk
    if world == 1 and not args.no_cpu_baseline:
        def gpu_check(kn, wn, C_oracle, f2_oracle):
            s2 = ms.Sketch(t=t, m=m, k=4, b=61, c=1, seed=args.seed, mode=mode)
            s2.update(torch.from_numpy(kn.view(np.int64)).to(dev),
                      None if wn is None else torch.from_numpy(wn).to(dev))
            return (np.array_equal(s2.counters().cpu().numpy(), C_oracle)
                    and s2.f2() == f2_oracle)
        line["cpu_baseline"] = cpu_baseline(wl, args.seed, args.cpu_seconds, gpu_check)
    if world == 1 and not args.no_extra and args.workload == "large" and args.keys == 0:
        # the other two figures of the metric ("% roofline; batched vs plain"),
        # each timed with its own clock record
        del keys, w, sk
        torch.cuda.empty_cache()
        line["plain_2p28"] = plain_result(args, ms, peaks, hbm_gbs, hbm_src)
        line["plain_2p20"] = plain_result(args, ms, peaks, hbm_gbs, hbm_src, "plain")
        line["batched"] = batched_result(args, ms, peaks)
    if world > 1:
        dist.destroy_process_group()
    return line


# ------------------------------------------------------------------ reference arm

def run_reference(args, wl):
    """The CPU oracle timed as the reference arm: K timed steps, each the oracle
    over the same bounded sample of the workload's stream (all host cores),
    sized so that the whole run takes about a minute and a half."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    coeffs = oracle.sketch_coeffs(61, 1, 4, wl["t"], wl["mode"], args.seed)
    kc, wc = make_inputs(wl, args.seed, 0, 1 << 16)
    t0 = time.perf_counter()
    oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, kc, wc, nthreads=cores)
    rate = (1 << 16) / max(time.perf_counter() - t0, 1e-6)
    per_step = max(0.05, min(args.cpu_seconds, 90.0 / max(1, args.steps)))
    n = int(min(wl["n"], max(1 << 12, rate * per_step)))
    n = 1 << int(math.log2(n))
    keys, w = make_inputs(wl, args.seed, 0, n)
    for _ in range(max(0, args.warmup)):
        oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, keys[:4096],
                         None if w is None else w[:4096], nthreads=cores)
    total = 0.0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        C = oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, keys, w,
                             nthreads=cores)
        oracle.f2_estimate(C)
        total += time.perf_counter() - t0
    steps = max(1, args.steps)
    value = n * steps / total
    sample = ("first %d keys of the same seeded stream per step, %d steps, %.1f s total on %d "
              "threads" % (n, steps, total, cores))
    return {
        "impl": "reference",
        "metric": "Count Sketch key updates/s (k=4, p=2^61-1)",
        "value": value,
        "unit": "keys/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": total / steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "inputs": inputs_desc(wl), "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "note": "the method has no reference implementation; this arm is the plain CPU oracle "
                "(unsigned __int128 % and /) on a bounded sample of the same stream",
    }


# ------------------------------------------------------------------ extra workloads

def _timed(fn, steps, warmup, stream=None):
    """Mean ms of fn() over `steps` runs after `warmup`, by CUDA events."""
    import torch
    for _ in range(max(1, warmup)):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _line(metric, value, unit, args, config, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "dtype": "u64", "data": "synthetic", "config": config}
    d.update(extra)
    return d


def run_sweep(args):
    """Prime-width sweep: 2^30 random keys, k=4, t=5, m=4096, unit weights, for
    p = 2^31-1 (u32 keys), 2^61-1 (u64), 2^89-1 (two-limb keys), 2^64-59 (u64)."""
    import torch
    import paper_2008_08654_gb300 as ms
    n = args.keys or (1 << 30)
    mul_rate, _ = ms.probe_mul128(variant=0, iters=1 << 12)
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for (b, c) in ms.PRIMES:
        p = (1 << b) - c
        if b == 31:
            keys = torch.from_numpy(datagen.u32_below(args.seed, p, n).view(np.int32)).cuda()
        elif b == 89:
            keys = torch.from_numpy(datagen.p89_keys(args.seed, n).view(np.int64)).cuda()
        else:
            keys = torch.from_numpy(datagen.u64_below(args.seed, p, n).view(np.int64)).cuda()
        sk = ms.Sketch(t=5, m=4096, k=4, b=b, c=c, seed=args.seed)

        def step():
            sk.reset()
            sk.update(keys)
        t = _timed(step, max(1, args.steps), args.warmup)
        kps = n / (t * 1e-3)
        res["2^%d-%d" % (b, c)] = {"keys_per_s": kps, "ms_per_step": t,
                                   "mul128_frac": kps * 15 / mul_rate,
                                   "launch": sk.last_launch(),
                                   "key_bytes": {31: 4, 61: 8, 89: 16, 64: 8}[b]}
        del keys, sk
        torch.cuda.empty_cache()
    clk = clocks.stop()
    best = res["2^61-1"]["keys_per_s"]
    return _line("Count Sketch key updates/s across primes (k=4, t=5, m=4096)", best, "keys/s",
                 args, {"workload": "prime sweep: %d random keys below p per prime, unit weights"
                        % n, "value_is": "p=2^61-1"},
                 per_prime=res, probe_mul64x64_per_s=mul_rate, **({"clocks": clk} if clk else {}))


def run_div(args):
    """ms_div microbenchmark: 2^30 uniform values below 2^122, p = 2^61-1; reads
    16 B and writes a 16-byte quotient and an 8-byte remainder per value."""
    import torch
    import paper_2008_08654_gb300 as ms
    n = args.keys or (1 << 30)
    v = datagen.u128_bits(args.seed, 122, n, stream=datagen.STREAM_VALUES)
    vd = torch.from_numpy(v.view(np.int64)).cuda()
    q = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    r = torch.empty(n, dtype=torch.int64, device="cuda")
    t = _timed(lambda: ms.div(61, 1, vd, q, r), max(1, args.steps), args.warmup)
    gbs = 40.0 * n / (t * 1e-3) / 1e9
    hbm_peak = 6787.9
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    return _line("ms_div values/s (p=2^61-1, v < 2^122)", n / (t * 1e-3), "values/s", args,
                 {"workload": "%d uniform 122-bit values, quotient (16 B) and remainder (8 B)" % n},
                 ms_per_step=t, roofline={"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                          "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
                                          "kernel": "k_divmod", "bytes_per_value": 40},
                 parity="tests/test_gpu_parity.py, tests/test_gpu_full.py")


# Table 2 (Sec. 5): ms for 10^7 divisions of 2b-bit values by 2^b - 1 on one
# core of an i7-8850H / a Xeon E5-2690 v4 (Algorithm division-generalized on GMP).
TABLE2_CPU_MS = {32: (138, 149), 64: (142, 198), 128: (157, 207), 256: (187, 222),
                 512: (291, 294), 1024: (358, 372)}


def run_divwide(args):
    """Table 2's workload on the GPU: 10^7 divisions of uniform 2b-bit values by
    p = 2^b - 1 for b in {32, 64, ..., 1024} (ms_div_wide).  Reads 2b bits and
    writes the (b+1)-bit quotient and b-bit remainder per value."""
    import torch
    import paper_2008_08654_gb300 as ms
    n = args.keys or 10 ** 7
    hbm_peak = 6787.9
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    rows, last = {}, None
    for b in (32, 64, 128, 256, 512, 1024):
        lv, lq, lr = (2 * b + 63) // 64, (b + 64) // 64, (b + 63) // 64
        v = datagen.u64_below(args.seed + b, 0, n * lv, stream=datagen.STREAM_VALUES).reshape(n, lv)
        if (2 * b) % 64:
            v[:, -1] &= np.uint64((1 << ((2 * b) % 64)) - 1)
        vd = torch.from_numpy(v.view(np.int64)).cuda()
        q = torch.empty((n, lq), dtype=torch.int64, device="cuda")
        r = torch.empty((n, lr), dtype=torch.int64, device="cuda")
        t = _timed(lambda: ms.div_wide(b, 1, vd, q=q, r=r), max(1, args.steps), args.warmup)
        nbytes = 8 * (lv + lq + lr)
        gbs = nbytes * n / (t * 1e-3) / 1e9
        rows["b=%d" % b] = {"ms_per_1e7": t * 1e7 / n, "values_per_s": n / (t * 1e-3),
                            "bytes_per_value": nbytes, "gbs": gbs, "hbm_frac": gbs / hbm_peak,
                            "paper_cpu_ms_per_1e7": list(TABLE2_CPU_MS[b])}
        last = (t, gbs, nbytes)
        del vd, q, r
        torch.cuda.empty_cache()
    t, gbs, nbytes = last
    return _line("wide ms_div values/s (b=1024, p=2^1024-1)", n / (t * 1e-3), "values/s", args,
                 {"workload": "%d uniform 2b-bit values per b, b in {32..1024}, p = 2^b - 1" % n,
                  "l2": "every b's inputs plus outputs exceed the 129 MB L2; no flush"},
                 ms_per_step=t, roofline={"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                          "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
                                          "kernel": "k_divwide", "bytes_per_value": nbytes},
                 table2=rows, parity="tests/test_gpu_divwide.py")


def run_query(args):
    """Point queries (the f_x estimate, Sec. 1.3): the large sketch (t=7, m=2^16,
    two-for-one) filled with its 2^28-key Zipf stream, then the estimates of
    2^26 keys of the same stream (8 B in, 8 B out per key; t rows hashed and t
    counters gathered per key, then their median)."""
    import torch
    import paper_2008_08654_gb300 as ms
    wl = WORKLOADS["large"]
    keys_np, _ = make_inputs(wl, args.seed, 0)
    keys = torch.from_numpy(keys_np.view(np.int64)).cuda()
    sk = ms.Sketch(t=wl["t"], m=wl["m"], k=4, b=61, c=1, seed=args.seed, mode=0)
    sk.update(keys)
    nq = args.keys or (1 << 26)
    q = keys[:nq].clone()
    del keys, keys_np
    torch.cuda.empty_cache()
    out = torch.empty(nq, dtype=torch.int64, device="cuda")
    peaks = probe_peaks(ms)
    hbm_gbs, hbm_src = hbm_peak_gbs()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t = _timed(lambda: sk.point_query(q, out), max(3, args.steps), max(3, args.warmup))
    clk = clocks.stop()
    roof = roofline_8d(nq, wl["t"], 1, 16, t * 1e-3, peaks, hbm_gbs, hbm_src)
    roof["kernel"] = "k_cs_point_query"
    line = _line("point queries/s (t=7, m=2^16, p=2^61-1)", nq / (t * 1e-3), "queries/s", args,
                 {"workload": "%d point queries of the 2^28-key Zipf(1.1) stream's first keys "
                              "on the large sketch (t=7, m=2^16) filled with that stream" % nq,
                  "l2": "queried keys (%d MiB) exceed the 129 MB L2; no flush" % (nq * 8 >> 20)},
                 ms_per_step=t, roofline=roof,
                 parity="tests/test_gpu_parity.py, tests/test_gpu_anyr.py")
    if clk:
        line["clocks"] = clk
    return line


def run_table1(args):
    """The paper's Table 1 workload: 10^7 k-universal hashes of random 64-bit
    keys for k in {2, 4, 8}, p = 2^61-1 and p = 2^89-1 (keys in device memory)."""
    import torch
    import paper_2008_08654_gb300 as ms
    n = args.keys or 10 ** 7
    k64 = datagen.u64_below(args.seed, (1 << 61) - 1, n)
    k89 = np.zeros((n, 2), dtype=np.uint64)
    k89[:, 0] = datagen.u64_below(args.seed + 1, 0, n)
    dev = {61: torch.from_numpy(k64.view(np.int64)).cuda(),
           89: torch.from_numpy(k89.view(np.int64)).cuda()}
    rows = {}
    for b in (61, 89):
        for k in (2, 4, 8):
            h = ms.Hash(k=k, b=b, c=1, seed=args.seed + k)
            out = h.out_tensor(n)
            t = _timed(lambda: h.eval(dev[b], out), max(1, args.steps), args.warmup)
            rows["p=2^%d-1,k=%d" % (b, k)] = {"ms_per_1e7_hashes": t * 1e7 / n,
                                              "hashes_per_s": n / (t * 1e-3)}
    return _line("k-universal hashes/s (p=2^61-1, k=4)", rows["p=2^61-1,k=4"]["hashes_per_s"],
                 "hashes/s", args, {"workload": "%d random 64-bit keys per (p, k)" % n},
                 table1=rows, parity="tests/test_gpu_parity.py, tests/test_gpu_full.py",
                 paper_cpu_ms_per_1e7={"p=2^61-1,k=4": [31.6, 34.3, 41.9],
                                       "p=2^89-1,k=4": [65.7, 68.7, 85.2]})


def batched_result(args, ms, peaks=None) -> dict:
    """Batched: independent sketches (t=5, m from {256, 1024, 4096, 8192}, own
    seeds, n_i = floor(10^(3+4U)) keys below 2^61-1, int32 weights in [-100, 100])
    in one persistent graph-captured launch, against one cs_update per sketch.
    The tuner picks the launch configuration for the whole plan, and once more
    for the sketches of each width class alone."""
    import torch
    S = args.sketches
    u = datagen.unit_doubles(args.seed, S, datagen.STREAM_LENGTHS)
    ns = np.floor(10.0 ** (3.0 + 4.0 * u)).astype(np.int64)
    widths = np.array([256, 1024, 4096, 8192])[
        datagen.u64_below(args.seed, 4, S, stream=datagen.STREAM_WIDTHS).astype(np.int64)]
    total = int(ns.sum())
    keys = torch.empty(total, dtype=torch.int64, device="cuda")
    wts = torch.empty(total, dtype=torch.int32, device="cuda")
    offs = np.concatenate([[0], np.cumsum(ns)])
    sketches, jobs = [], []
    for i in range(S):
        s0 = args.seed * 7919 + i
        a, b = int(offs[i]), int(offs[i + 1])
        keys[a:b].copy_(torch.from_numpy(datagen.u64_below(s0, (1 << 61) - 1, b - a)
                                         .view(np.int64)))
        wts[a:b].copy_(torch.from_numpy(datagen.i32_range(s0, -100, 100, b - a)))
        sk = ms.Sketch(t=5, m=int(widths[i]), k=4, seed=s0)
        sketches.append(sk)
        jobs.append((sk, keys[a:b], wts[a:b]))
    cands = []
    for threads in (256, 512, 1024):
        for chunk in (1 << 15, 1 << 17, 1 << 19):
            for ratio in (2, 8, 32):
                cands.append({"threads": threads, "chunk_keys": chunk, "smem_min_ratio": ratio})
    per_m = {}
    if args.no_tune:
        best, times, ncand = ms.default_tuning().as_dict(), [], 0
    else:
        best, times = ms.tune_batched(jobs, cands, reps=2)
        ncand = len(cands)
        for mc in (256, 1024, 4096, 8192):
            sub = [j for j, wd in zip(jobs, widths) if wd == mc]
            if not sub:
                continue
            b_m, t_m = ms.tune_batched(sub, cands, reps=2)
            keys_m = int(sum(j[1].numel() for j in sub))
            per_m[str(mc)] = {"sketches": len(sub), "keys": keys_m, "choice": b_m,
                              "best_ms": min(t_m) if t_m else None,
                              "keys_per_s": keys_m / (min(t_m) * 1e-3) if t_m else None}
    plan = ms.Batch(jobs, best)

    def reset_all():
        for sk in sketches:
            sk.reset()

    def plain():
        for sk, kk, ww in jobs:
            sk.update(kk, ww)

    reset_all()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t_graph = _timed(plan.launch, max(3, args.steps), max(3, args.warmup))
    t_direct = _timed(plan.launch_direct, max(3, args.steps), 3)
    t_plain = _timed(plain, max(3, min(args.steps, 5)), 3)
    clk = clocks.stop()
    # the batched plan and the separate launches give the same counters on a
    # sample of sketches (parity with the oracle: tests/test_gpu_batched.py)
    sample = list(range(0, S, max(1, S // 6)))[:6]
    reset_all()
    plan.launch()
    torch.cuda.synchronize()
    got = [sketches[i].counters().cpu().numpy() for i in sample]
    reset_all()
    for i in sample:
        sk, kk, ww = jobs[i]
        sk.update(kk, ww)
    torch.cuda.synchronize()
    same = all(np.array_equal(g, sketches[i].counters().cpu().numpy()) for g, i in zip(got, sample))
    info = plan.info()
    out = {"workload": "%d sketches, %d keys in total (log-uniform 1e3..1e7 per sketch), t=5, "
                       "m uniform over {256, 1024, 4096, 8192}, weights in [-100, 100]"
                       % (S, total),
           "value": total / (t_graph * 1e-3), "unit": "keys/s", "ms_per_step": t_graph,
           "keys": total,
           "m_classes": {str(mc): int((widths == mc).sum()) for mc in (256, 1024, 4096, 8192)},
           "direct_launch_keys_per_s": total / (t_direct * 1e-3),
           "plain_launches_keys_per_s": total / (t_plain * 1e-3),
           "plain_launches_ms": t_plain,
           "speedup_vs_plain_launches": t_plain / t_graph, "tuner_choice": best,
           "tuner_choice_per_m": per_m, "tuner_candidates": ncand, "tuner_times_ms": times,
           "plan": info, "same_as_plain_launches_on_sample": bool(same),
           "gpu_launches_per_step": 2}
    if peaks:
        out["mul128_frac"] = total * 15 / (t_graph * 1e-3) / peaks["mul128_per_s"]
    if clk:
        out["clocks"] = clk
    del plan, jobs, sketches, keys, wts
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    import paper_2008_08654_gb300 as ms
    r = batched_result(args, ms, probe_peaks(ms))
    extra = {k: v for k, v in r.items() if k not in ("workload", "value", "unit")}
    return _line("batched Count Sketch key updates/s (k=4, p=2^61-1, t=5)", r["value"], "keys/s",
                 args, {"workload": r["workload"], "m_classes": r["m_classes"]}, **extra)


def run_serving(args):
    """Serving: device-resident sketches (t=5, k=4, p=2^61-1, m uniform over
    {1024, 4096}); Poisson arrivals mixing updates (log-uniform 256..2^20 Zipf(1.1)
    keys, unit weights) with F2 queries (10%); 40 GB staging budget.  First a
    saturating run measures peak keys/s, then offered loads of 50/80/95% of it."""
    import torch
    import paper_2008_08654_gb300 as ms
    S = args.sketches if args.sketches != 4096 else 10000
    widths = [1024 if x == 0 else 4096
              for x in datagen.u64_below(args.seed, 2, S, stream=datagen.STREAM_WIDTHS)]
    srv = ms.Server(widths, t=5, seed_base=args.seed, staging_bytes=40 << 30, max_inflight=4096,
                    max_batch_keys=1 << 25, max_batch_requests=4096, timeout_s=120.0)
    # 2^26 keys (512 MiB, larger than the L2): page-locked, so the update kernel
    # reads each request's keys in place over the host link
    pool = torch.from_numpy(datagen.zipf(args.seed, 1.1, 1 << 32, 1 << 26).view(np.int64))
    pool = pool.pin_memory()
    # 2e5 requests per run (each of the 10^4 sketches about 20 times): windows
    # of more than a second at every offered load
    count = max(200, args.keys or 200000)
    qf, lo, hi = 0.1, 256, 1 << 20
    mean_n = (hi - lo) / math.log(hi / lo)
    srv.run_load(pool, count=2000, rate_per_s=1e6, query_fraction=qf, min_keys=lo, max_keys=hi,
                 seed=args.seed + 99)  # warm-up

    def measured(rate, seed):
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        r = srv.run_load(pool, count=count, rate_per_s=rate, query_fraction=qf, min_keys=lo,
                         max_keys=hi, seed=seed)
        clk = clocks.stop()
        if clk:
            r["clocks"] = clk
        return r

    peak = measured(1e7, args.seed)
    levels = {}
    for frac in (0.5, 0.8, 0.95):
        rate = frac * peak["keys_per_s"] / ((1 - qf) * mean_n)
        levels["%d%%" % int(frac * 100)] = measured(rate, args.seed + int(frac * 100))
    srv.close()
    return _line("served Count Sketch key updates/s (k=4, p=2^61-1, t=5)", peak["keys_per_s"],
                 "keys/s", args,
                 {"workload": "%d device-resident sketches, m in {1024, 4096}; %d requests per "
                              "run, 10%% F2 queries, updates of log-uniform 256..2^20 Zipf(1.1) "
                              "keys from a page-locked host pool of 2^26 keys (512 MiB), read in place by "
                              "the update kernel; 40 GB staging" % (S, count)},
                 saturated=peak, offered_load=levels,
                 **({"clocks": peak["clocks"]} if "clocks" in peak else {}))


EXTRA = {"sweep": run_sweep, "div": run_div, "divwide": run_divwide, "table1": run_table1,
         "batched": run_batched, "query": run_query,
         "serving": run_serving}


def main():
    args = parse_args()
    if args.workload in EXTRA:
        line = EXTRA[args.workload](args)
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")
        return
    wl = dict(WORKLOADS[args.workload])
    if args.keys > 0:
        wl["n"] = args.keys
        wl["desc"] = wl["desc"] + " (reduced to %d keys)" % args.keys
    if args.impl == "reference":
        line = run_reference(args, wl)
    else:
        line = run_ours(args, wl)
    if line is not None:
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")


if __name__ == "__main__":
    main()
