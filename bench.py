#!/usr/bin/env python
"""Benchmark: in-place Smoothed Striding partition of 2^30 uint64 keys on one GB300.

Workload (default): n = 2^30 uniform uint64 keys (8 GiB) from SplitMix64, pivot
2^63 - 1 (about half the keys are predecessors), Recursive Smoothed Striding
through the C ABI (lp_partition_u64_async).  Each step regenerates the input
on the device (untimed; it also flushes L2, the input being 8 GiB) and times
the partition with CUDA events on the launching stream.

value   = effective GB/s = 3 * 8 bytes * n / partition time (the "2 reads + 1
          write of the key bytes" convention), summed over ranks.
roofline: the dominant kernel is the level-0 Partial Partition Step; its
          algorithmic traffic is one read and one write of every key in its
          range (2 * 8 * n bytes), timed live with the library's per-level
          CUDA events, against the measured HBM copy bandwidth.
e2e     = the same metric through the C ABI with host buffers: pinned host ->
          device copy of the keys, partition, device -> host copy of the
          partitioned keys and the split, all inside the timed region.
cpu_baseline: the serial CPU oracle (two-pointer partition) on a bounded
          sample of the same workload, on one host core.

--impl reference runs the oracle alone (the reference arm of this repo: the
paper's method has no GPU reference), on host cores, same metric and config.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2004_12532_gb300 import inputs  # noqa: E402

METRIC = "in-place partition GB/s (uint64, n=2^30)"
UNIT = "GB/s"
KERNEL_SOURCES = ["lp_smoothed.cuh", "lp_kernels.cu", "lp_plan.h", "lp_device.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, default=None,
                    help="default 30 (u64), 31 (u32), 29 (kv)")
    ap.add_argument("--dtype", choices=["u64", "u32", "kv"], default="u64")
    ap.add_argument("--quantile", type=int, default=50, help="percent of keys <= pivot")
    ap.add_argument("--variant", choices=["smoothed", "strided", "lowspace", "hybrid"],
                    default="smoothed")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--seed", type=int, default=0xC0FF2)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2004_12532_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(n_keys):
    """dram read+write bytes per level-0 launch from the committed ncu summary,
    scaled to n_keys, if the summary was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "partition_kernel_u64_ncu.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    try:
        per_key = float(kv["dram_bytes_per_key"])
    except (KeyError, ValueError):
        return None
    return per_key * n_keys


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r[0] for r in rows] or [0.0]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_gbs(log2n_sample, pivot, seed, min_seconds=8.0, max_reps=5):
    import oracle
    n = 1 << log2n_sample
    times = []
    t_start = time.time()
    for r in range(max_reps):
        a = inputs.uniform_u64(n, seed + r)
        t0 = time.perf_counter()
        oracle.partition(a, pivot)
        times.append(time.perf_counter() - t0)
        if time.time() - t_start > min_seconds and len(times) >= 2:
            break
    med = statistics.median(times)
    return 3 * 8 * n / med / 1e9, n, len(times), med


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    pivot = inputs.quantile_pivot(1, 2)
    log2s = min(args.log2n, 26)
    n = 1 << log2s
    for w in range(args.warmup):
        a = inputs.uniform_u64(n, args.seed + 1000 + w)
        oracle.partition(a, pivot)
    total = 0.0
    for k in range(args.steps):
        a = inputs.uniform_u64(n, args.seed + k)
        t0 = time.perf_counter()
        oracle.partition(a, pivot)
        total += time.perf_counter() - t0
    ms = total / args.steps * 1e3
    value = 3 * 8 * n / (ms / 1e3) / 1e9
    sample = "2^%d uint64 keys per step (of the 2^%d workload), same distribution and pivot" % (
        log2s, args.log2n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "partition u64 n=2^%d pivot=2^63-1 (50%%)" % args.log2n,
                   "oracle": "serial two-pointer partition (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2004_12532_gb300 import binding as lp

    n = 1 << args.log2n
    dt = args.dtype
    K = 4 if dt == "u32" else 8          # key bytes
    E = 16 if dt == "kv" else K          # bytes moved per key (key + payload)
    pivot = inputs.quantile_pivot(args.quantile, 100, 32 if dt == "u32" else 64)
    variant = {"smoothed": lp.LP_SMOOTHED, "strided": lp.LP_STRIDED,
               "lowspace": lp.LP_LOWSPACE, "hybrid": lp.LP_HYBRID}[args.variant]
    keys = torch.empty(n, dtype=torch.int32 if dt == "u32" else torch.int64, device="cuda")
    vals = torch.empty(n, dtype=torch.int64, device="cuda") if dt == "kv" else None
    d_split = torch.zeros(1, dtype=torch.int64, device="cuda")

    def fill(seed):
        if dt == "u32":
            lp.lp_fill_uniform_u32(keys, seed)
        else:
            lp.lp_fill_uniform_u64(keys, seed)
        if vals is not None:
            lp.lp_fill_iota_u64(vals)

    def part(seed):
        if dt == "u32":
            lp.lp_partition_u32_async(ctx, keys, pivot, d_split, variant, seed=seed)
        elif dt == "kv":
            lp.lp_partition_kv_u64_async(ctx, keys, vals, pivot, d_split, variant, seed=seed)
        else:
            lp.lp_partition_u64_async(ctx, keys, pivot, d_split, variant, seed=seed)
    ctx = lp.Ctx(local)
    ctx.set_timing(True)
    stream = torch.cuda.current_stream()
    seed0 = args.seed + 7919 * rank

    for w in range(args.warmup):
        fill(seed0 + 100000 + w)
        part(w)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    part_ms, lvl0_ms, lvl0_n, launches, traffic_keys, kern_ms = [], [], [], 0, [], []
    levels_seen, level_ms = [], []
    barrier()
    wall0 = time.perf_counter()
    clocks.start()
    for k in range(args.steps):
        fill(seed0 + k)
        ev0.record(stream)
        part(k)
        ev1.record(stream)
        ev1.synchronize()
        part_ms.append(ev0.elapsed_time(ev1))
        launches += ctx.last_launches
        st = ctx.level_stats()
        kern_ms.append(ctx.kernel_ms())
        lvl0_ms.append(st[0][4])
        lvl0_n.append(st[0][1] - st[0][0])
        traffic_keys.append(sum(hi - lo for lo, hi, _, _, _ in st))
        levels_seen.append([(hi - lo) for lo, hi, _, _, _ in st if hi > lo])
        level_ms.append([ms_ for _, _, _, _, ms_ in st])
    barrier()
    wall_s = time.perf_counter() - wall0
    clk = clocks.stop()
    t = int(d_split.item())

    ms = sum(part_ms) / len(part_ms)
    ms_all = ms
    if ws > 1:
        import torch.distributed as dist
        x = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        ms_all = float(x.item())
    value = ws * 3 * E * n / (ms_all / 1e3) / 1e9

    peak, peak_kind = measured_peaks()
    k_ms = sum(kern_ms) / len(kern_ms)
    k_keys = sum(traffic_keys) / len(traffic_keys)
    k_bytes = 2 * E * k_keys  # one read and one write of every key of every level
    achieved = k_bytes / (k_ms / 1e3) / 1e9
    traffic = profiled_traffic(k_keys) if dt == "u64" else None
    l0_ms = sum(lvl0_ms) / len(lvl0_ms)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "partition_kernel<%s> (all levels, one cooperative launch)" % (
                    {"u64": "uint64_t", "u32": "uint32_t", "kv": "uint64_t, payload"}[dt]),
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": k_bytes,
                "ms_per_launch": k_ms,
                "level0_gbs_device_timestamps": 2 * E * (sum(lvl0_n) / len(lvl0_n)) /
                (l0_ms / 1e3) / 1e9 if l0_ms > 0 else None}

    metric = METRIC if (dt == "u64" and args.log2n == 30) else \
        "in-place partition GB/s (%s, n=2^%d)" % ({"u64": "uint64", "u32": "uint32",
                                                   "kv": "uint64 key + uint64 payload"}[dt],
                                                  args.log2n)
    result = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if dt == "u32" else "u64",
        "data": "synthetic (SplitMix64 uniform keys, seeded)",
        "config": {"workload": "partition %s n=2^%d pivot at %d%% quantile, %s" % (
                       dt, args.log2n, args.quantile, args.variant),
                   "n": n, "pivot": pivot, "variant": args.variant, "dtype": dt,
                   "l2": "inputs larger than L2 (8 GiB), regenerated on device between steps",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline,
        "gpu_launches": launches,
        "split_last_step": t,
        "true_gbs": ws * 2 * K * (sum(traffic_keys) / len(traffic_keys)) / (ms_all / 1e3) / 1e9,
        "level_ranges_last_step": levels_seen[-1],
        "level_ms_mean": [round(sum(x) / len(x), 4) for x in zip(*level_ms)],
        "aux_bytes": ctx.aux_bytes,
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk

    if not args.no_e2e and dt == "u64":
        result["e2e"] = e2e_leg(args, lp, ctx, keys, d_split, pivot, variant, n, seed0, stream)
    if rank == 0 and ws == 1 and not args.no_cpu and dt == "u64":
        gbs, ns, reps, med = cpu_oracle_gbs(min(args.log2n, 27), pivot, args.seed)
        result["cpu_baseline"] = {
            "value": gbs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "2^%d uint64 keys, same distribution and pivot, median of %d runs "
                      "(%.2f s each) of the serial two-pointer partition" % (
                          int(np.log2(ns)), reps, med),
            "host_cores_available": os.cpu_count()}
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def e2e_leg(args, lp, ctx, keys, d_split, pivot, variant, n, seed0, stream):
    import torch
    host_in = torch.empty(n, dtype=torch.int64, pin_memory=True)
    host_out = torch.empty(n, dtype=torch.int64, pin_memory=True)
    host_split = torch.empty(1, dtype=torch.int64, pin_memory=True)
    lp.lp_fill_uniform_u64(keys, seed0 + 555)
    host_in.copy_(keys)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    for k in range(max(1, args.e2e_steps)):
        ev0.record(stream)
        keys.copy_(host_in, non_blocking=True)
        lp.lp_partition_u64_async(ctx, keys, pivot, d_split, variant, seed=k)
        host_out.copy_(keys, non_blocking=True)
        host_split.copy_(d_split, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    ms = sum(times) / len(times)
    return {"value": 3 * 8 * n / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n + 8,
            "path": "pinned host -> device, lp_partition_u64_async, device -> pinned host"}


def main():
    args = parse()
    if args.log2n is None:
        args.log2n = {"u64": 30, "u32": 31, "kv": 29}[args.dtype]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
