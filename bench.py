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
e2e     = the same metric through the C ABI with a host buffer:
          lp_partition_host_u64 partitions a pinned host array in place
          (chunked uploads, device partitions and copies back, overlapping),
          all inside the timed region.  (--workload quicksort / batched: a
          pinned host -> device copy, the device call, a device -> host copy.)
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
    ap.add_argument("--variant", choices=["smoothed", "strided", "lowspace", "hybrid",
                                          "implicit"],
                    default="smoothed")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-yardstick", action="store_true",
                    help="skip the out-of-place library partition timed beside ours")
    ap.add_argument("--seed", type=int, default=0xC0FF2)
    ap.add_argument("--workload", choices=["partition", "quicksort", "batched", "serve"],
                    default="partition",
                    help="partition (default): one 2^30-key partition; quicksort: 2^28 uint64 "
                         "sort; batched: 4096 partitions of log-uniform sizes in one graph; "
                         "serve: Poisson stream of partition and sort requests")
    ap.add_argument("--pivot-samples", type=int, choices=[3, 15], default=3,
                    help="quicksort: pivot = median of this many seeded keys (3 per the "
                         "workload's definition)")
    ap.add_argument("--input", choices=["uniform", "sorted", "reverse", "dup16"],
                    default="uniform", help="quicksort input")
    ap.add_argument("--instances", type=int, default=4096, help="batched: instance count")
    ap.add_argument("--min-chunks", type=int, default=0,
                    help="quicksort: lines per group, at least, of the batched steps (0: default)")
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests per step")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: mean arrivals per s")
    ap.add_argument("--budget-gib", type=float, default=64.0, help="serve: HBM budget")
    ap.add_argument("--slots", type=int, default=256, help="serve: requests in flight, at most")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_hash():
    """Hash of the partition kernel's sources without // comments and blank
    lines (a comment changes no kernel)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        for line in open(os.path.join(ROOT, "paper_2004_12532_gb300", "csrc", f), "rb"):
            code = line.split(b"//", 1)[0].rstrip()
            if code:
                h.update(code + b"\n")
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


def cpu_parallel_gbs(log2n, pivot, seed, reps=3):
    """The Smoothed Striding partition on all host cores (OpenMP, libcpuyard.so):
    the paper's own multicore setting, as a second CPU baseline."""
    import ctypes
    path = os.path.join(ROOT, "paper_2004_12532_gb300", "libcpuyard.so")
    if not os.path.exists(path):
        return {"unavailable": "libcpuyard.so not built"}
    L = ctypes.CDLL(path)
    L.cy_smoothed_partition_u64.restype = ctypes.c_uint64
    L.cy_smoothed_partition_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_int, ctypes.c_uint64]
    n = 1 << log2n
    threads = os.cpu_count() or 1
    times, ok = [], True
    for r in range(reps):
        a = inputs.uniform_u64(n, seed + r)
        want = int(np.count_nonzero(a <= np.uint64(pivot)))
        t0 = time.perf_counter()
        t = L.cy_smoothed_partition_u64(a.ctypes.data, n, pivot, threads, seed + r)
        times.append(time.perf_counter() - t0)
        ok = ok and t == want and bool(np.all(a[:t] <= np.uint64(pivot))) and \
            bool(np.all(a[t:] > np.uint64(pivot)))
    med = statistics.median(times)
    return {"value": 3 * 8 * n / med / 1e9, "unit": "GB/s", "cores": threads,
            "kind": "Smoothed Striding on the host cores (OpenMP)",
            "sample": "2^%d uint64 keys, same distribution and pivot, median of %d runs" % (
                log2n, reps), "correct": ok}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "quicksort":
        return run_reference_sort(args)
    if args.workload == "batched":
        return run_reference_batched(args)
    if args.workload == "serve":
        return run_reference_serve(args)
    import oracle
    if args.dtype != "u64":
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm times uint64 partitions only"}))
        return
    pivot = inputs.quantile_pivot(args.quantile, 100, 64)
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
        "config": {"workload": "partition u64 n=2^%d pivot at %d%% quantile, %s" % (
                       args.log2n, args.quantile, args.variant),
                   "n": 1 << args.log2n, "pivot": pivot, "variant": args.variant,
                   "dtype": "u64", "oracle": "serial two-pointer partition (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def reference_line(args, metric, value, unit, ms, workload, oracle_kind, sample, dtype="u64"):
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": {"workload": workload, "oracle": oracle_kind},
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_reference_sort(args):
    import oracle
    log2s = min(args.log2n, 22)
    n = 1 << log2s
    for w in range(args.warmup):
        oracle.quicksort(host_sort_input(args.input, n, args.seed + 1000 + w), w)
    total = 0.0
    for k in range(args.steps):
        a = host_sort_input(args.input, n, args.seed + k)
        t0 = time.perf_counter()
        oracle.quicksort(a, k)
        total += time.perf_counter() - t0
    ms = total / args.steps * 1e3
    reference_line(args, "quicksort keys/s (uint64, n=2^%d, %s)" % (args.log2n, args.input),
                   n / (ms / 1e3) / 1e9, "Gkeys/s", ms,
                   "quicksort u64 n=2^%d input=%s" % (args.log2n, args.input),
                   "serial quicksort (CPU)",
                   "2^%d uint64 keys per step, same input kind" % log2s)


def run_reference_batched(args):
    sizes, _, _ = batch_layout(args.instances, args.seed)
    keys_total = int(sum(int(m) for m in sizes))
    for w in range(args.warmup):
        cpu_oracle_batch(sizes[:8], args.seed + w, 0.5)
    vals = []
    keys = 0
    for k in range(args.steps):
        v, done, inst = cpu_oracle_batch(sizes, args.seed + k, 2.0)
        vals.append(v)
        keys += done
    v = statistics.mean(vals)
    ms = keys / args.steps / (v * 1e9) * 1e3
    reference_line(args, "batched partition keys/s (%d uint64 instances, sizes log-uniform "
                   "[2^8, 2^22])" % args.instances, v, "Gkeys/s", ms,
                   "batched partition, %d instances, %d keys in all" % (args.instances,
                                                                         keys_total),
                   "serial two-pointer partition per instance (CPU)",
                   "about 2 s of instances per step, in batch order")


def run_reference_serve(args):
    """The oracle serving the same request mix one request at a time on one host
    core (partition: two-pointer; sort: serial quicksort), on a bounded sample."""
    import oracle
    rng = np.random.default_rng(args.seed)
    sizes = inputs.log_uniform_sizes(4096, args.seed, 10, 26)
    vals, keys_all = [], 0
    for k in range(args.warmup + args.steps):
        spent, keys = 0.0, 0
        for i, m in enumerate(sizes):
            if spent > 1.0:
                break
            bits = 64 if rng.random() < 0.5 else 32
            a = inputs.uniform_u64(int(m), args.seed + i) if bits == 64 else \
                inputs.uniform_u32(int(m), args.seed + i)
            t0 = time.perf_counter()
            if rng.random() < 0.3:
                oracle.quicksort(a, i)
            else:
                oracle.partition(a, inputs.quantile_pivot(int(rng.integers(1, 100)), 100, bits))
            spent += time.perf_counter() - t0
            keys += int(m)
        if k >= args.warmup:
            vals.append(keys / spent / 1e9)
            keys_all += keys
    v = statistics.mean(vals)
    reference_line(args, "served keys/s (Poisson %.0f req/s, 70%% partition / 30%% sort, sizes "
                   "log-uniform [2^10, 2^26], uint32/uint64)" % args.rate, v, "Gkeys/s",
                   keys_all / args.steps / (v * 1e9) * 1e3,
                   "serve %d requests per step at %.0f req/s" % (args.requests, args.rate),
                   "serial partition / quicksort per request, one at a time",
                   "requests in stream order until 1 s of service time is spent (one large "
                   "sort can overrun it), service time only", dtype="u32+u64")


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
               "lowspace": lp.LP_LOWSPACE, "hybrid": lp.LP_HYBRID,
               "implicit": None}[args.variant]
    if variant is None and dt == "kv":
        raise SystemExit("--variant implicit: keys only")
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
        if variant is None:  # values kept in key order: its own entry point, split to host
            d_split.fill_(lp.lp_lowspace_implicit_partition(ctx, keys, pivot))
        elif dt == "u32":
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
    bytes_all, ms_all = whole_job(ws, 3 * E * n, ms)
    value = bytes_all / (ms_all / 1e3) / 1e9

    peak, peak_kind = measured_peaks()
    k_ms = sum(kern_ms) / len(kern_ms)
    k_keys = sum(traffic_keys) / len(traffic_keys)
    kname = {"u64": "uint64_t", "u32": "uint32_t", "kv": "uint64_t, payload"}[dt]
    basis = None
    if args.variant in ("lowspace", "implicit"):
        # Sec. 5's accounting of the low-space partition: 3.5 read/write passes
        # and 0.5 read pass over the keys, i.e. 7.5 key bytes per key -- derived
        # for about half predecessors; with a small minority the Reorder phase
        # moves few keys and the figure overstates the work (frac above 1)
        k_bytes = 7.5 * E * n
        basis = ("Sec. 5 bound: 7.5 key bytes per key for about half predecessors; "
                 "minority fraction of this run %.3f" % (min(t, n - t) / n if n else 0.0))
        kernel = "lowspace_kernel<%s%s> (all phases, one cooperative launch)" % (
            kname, ", values in key order" if variant is None else "")
        traffic = None
    else:
        k_bytes = 2 * E * k_keys  # one read and one write of every key of every level
        kernel = "partition_kernel<%s> (all levels, one cooperative launch)" % kname
        traffic = profiled_traffic(k_keys) if dt == "u64" and args.variant == "smoothed" \
            else None
    achieved = k_bytes / (k_ms / 1e3) / 1e9
    l0_ms = sum(lvl0_ms) / len(lvl0_ms)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": k_bytes,
                "ms_per_launch": k_ms,
                "level0_gbs_device_timestamps": 2 * E * (sum(lvl0_n) / len(lvl0_n)) /
                (l0_ms / 1e3) / 1e9 if l0_ms > 0 else None}
    if basis:
        roofline["basis"] = basis

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

    if not args.no_yardstick and dt == "u64":
        result["yardstick_cub"] = cub_yardstick(args, keys, n, pivot, stream, fill, seed0, t)
    if not args.no_e2e and dt == "u64" and args.variant == "smoothed":
        result["e2e"] = e2e_leg(args, lp, ctx, keys, d_split, pivot, variant, n, seed0, stream)
    if rank == 0 and ws == 1 and not args.no_cpu and dt == "u64":
        result["cpu_parallel"] = cpu_parallel_gbs(min(args.log2n, 27), pivot, args.seed)
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


def cub_yardstick(args, keys, n, pivot, stream, fill, seed0, split_ours):
    """The out-of-place library partition (CUB DevicePartition::If, built into
    libyardstick.so) of the same input, timed the same way: what giving up the
    in-place property buys at the same bandwidth.  Not the product path."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_2004_12532_gb300", "libyardstick.so")
    if not os.path.exists(path):
        return {"unavailable": "libyardstick.so not built"}
    L = ctypes.CDLL(path)
    tb = ctypes.c_size_t()
    if L.yd_cub_partition_temp_bytes(ctypes.c_uint64(n), ctypes.byref(tb)) != 0:
        return {"unavailable": "temp size query failed"}
    out = torch.empty_like(keys)
    tmp = torch.empty(max(1, tb.value), dtype=torch.uint8, device="cuda")
    sel = torch.zeros(1, dtype=torch.int64, device="cuda")
    L.yd_cub_partition_u64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    for k in range(max(3, args.warmup) + max(3, args.steps)):
        fill(seed0 + k)
        ev0.record(stream)
        rc = L.yd_cub_partition_u64(keys.data_ptr(), out.data_ptr(), n, pivot, sel.data_ptr(),
                                    tmp.data_ptr(), tb.value, stream.cuda_stream)
        ev1.record(stream)
        ev1.synchronize()
        if rc != 0:
            return {"unavailable": "cub partition failed"}
        if k >= max(3, args.warmup):
            times.append(ev0.elapsed_time(ev1))
    fill(seed0 + args.steps - 1)  # the last timed input of our partition, for the split
    L.yd_cub_partition_u64(keys.data_ptr(), out.data_ptr(), n, pivot, sel.data_ptr(),
                           tmp.data_ptr(), tb.value, stream.cuda_stream)
    torch.cuda.synchronize()
    ms = sum(times) / len(times)
    res = {"kernel": "cub::DevicePartition::If (out of place)", "ms_per_step": ms,
           "effective_gbs": 3 * 8 * n / (ms / 1e3) / 1e9,
           "read_write_gbs": 2 * 8 * n / (ms / 1e3) / 1e9,
           "extra_device_bytes": 8 * n + tb.value,
           "same_split": int(sel.item()) == split_ours}
    del out, tmp
    return res


def e2e_leg(args, lp, ctx, keys, d_split, pivot, variant, n, seed0, stream):
    """The same metric through the C ABI with a HOST buffer: every step hands
    lp_partition_host_u64 a pinned host array of n keys and gets it back
    partitioned in place (its uploads, device partitions and copies back all
    inside the timed region); the input is restored between steps, untimed.
    The Smoothed Striding variant only (the host call's device partition)."""
    import torch
    times, t, err = [], 0, None
    try:  # pinned memory may run short with many ranks per host: report, don't crash
        host_in = torch.empty(n, dtype=torch.int64, pin_memory=True)
        host_work = torch.empty(n, dtype=torch.int64, pin_memory=True)
        lp.lp_fill_uniform_u64(keys, seed0 + 555)
        host_in.copy_(keys)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for k in range(max(1, args.e2e_steps) + 1):  # the first call sizes the device copy
            host_work.copy_(host_in)
            torch.cuda.synchronize()
            ev0.record(stream)
            t = lp.lp_partition_host(ctx, host_work, pivot, seed=k, stream=stream)
            ev1.record(stream)
            ev1.synchronize()
            if k > 0:
                times.append(ev0.elapsed_time(ev1))
        del host_in, host_work
    except (RuntimeError, lp.LPError) as e:
        err = str(e).splitlines()[0][:200]
    ws = dist_env()[0]
    # every rank joins the reduction; a rank that failed brings an infinite time
    my_ms = sum(times) / len(times) if times and err is None else float("inf")
    bytes_all, ms = whole_job(ws, 3 * 8 * n, my_ms)  # every rank's array
    if not np.isfinite(ms):
        return {"value": None, "unit": UNIT,
                "unavailable": err or "another rank's end-to-end leg failed"}
    return {"value": bytes_all / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "ms_each_step": [round(x, 2) for x in times],
            "ms_median": float(np.median(times)),
            "h2d_bytes_per_step": 8 * n * ws, "d2h_bytes_per_step": 8 * n * ws, "split": t,
            "path": "lp_partition_host_u64 on a pinned host array (chunked uploads, "
                    "device partitions and copies back overlapping)"}


# ---------------------------------------------------------------- quicksort

def unsigned_order(t):
    """Signed view of uint64 bits whose order is the unsigned order (an involution)."""
    import torch
    return t ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=t.device)


def fill_sort_input(lp, keys, kind, seed):
    import torch
    lp.lp_fill_uniform_u64(keys, seed)
    if kind == "sorted":
        keys.copy_(unsigned_order(torch.sort(unsigned_order(keys)).values))
    elif kind == "reverse":
        keys.copy_(unsigned_order(torch.sort(unsigned_order(keys), descending=True).values))
    elif kind == "dup16":
        keys.bitwise_and_(15)


def host_sort_input(kind, n, seed):
    if kind == "uniform":
        return inputs.uniform_u64(n, seed)
    if kind == "sorted":
        return inputs.sorted_u64(n, seed)
    if kind == "reverse":
        return inputs.reverse_sorted_u64(n, seed)
    return inputs.heavy_duplicates_u64(n, seed, 16)


def cpu_oracle_sort(kind, log2n, seed, min_seconds=8.0, max_reps=5):
    import oracle
    n = 1 << log2n
    times = []
    t_start = time.time()
    for r in range(max_reps):
        a = host_sort_input(kind, n, seed + r)
        t0 = time.perf_counter()
        oracle.quicksort(a, r)
        times.append(time.perf_counter() - t0)
        if time.time() - t_start > min_seconds and len(times) >= 2:
            break
    med = statistics.median(times)
    return n / med / 1e9, n, len(times), med


def init_dist(local, ws):
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def whole_job(ws, units, ms):
    """(sum of units over ranks, max of ms over ranks): the whole-job work and
    its time.  Single process: (units, ms).  The reduction runs on the
    process group's device (CUDA under NCCL, the host under gloo)."""
    if ws == 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def run_quicksort(args):
    import torch
    ws, rank, local = dist_env()
    init_dist(local, ws)
    from paper_2004_12532_gb300 import binding as lp
    n = 1 << args.log2n
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    ctx = lp.Ctx(local)
    ctx.set_timing(True)
    if args.min_chunks:
        lp.lp_ctx_set_batch_tuning(ctx, min_chunks=args.min_chunks)
    stream = torch.cuda.current_stream()
    seed0 = args.seed + 7919 * rank
    for w in range(args.warmup):
        fill_sort_input(lp, keys, args.input, seed0 + 100000 + w)
        lp.lp_quicksort(ctx, keys, seed=w, pivot_samples=args.pivot_samples)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, stats, launches = [], [], 0
    wall0 = time.perf_counter()
    clocks.start()
    for k in range(args.steps):
        fill_sort_input(lp, keys, args.input, seed0 + k)  # untimed; 2 GiB > L2
        torch.cuda.synchronize()
        ev0.record(stream)
        lp.lp_quicksort(ctx, keys, seed=k, pivot_samples=args.pivot_samples)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        stats.append(ctx.sort_stats())
        launches += ctx.last_launches
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - wall0
    clk = clocks.stop()
    key = unsigned_order(keys)
    sorted_ok = bool((key[1:] >= key[:-1]).all())
    ms = sum(step_ms) / len(step_ms)
    keys_all, ms_all = whole_job(ws, n, ms)
    value = keys_all / (ms_all / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    pk = sum(s["partition_keys"] for s in stats) / len(stats)
    pms = sum(s["partition_ms"] for s in stats) / len(stats)
    sk = sum(s["sort_keys"] for s in stats) / len(stats)
    sms = sum(s["sort_ms"] for s in stats) / len(stats)
    achieved = 2 * 8 * pk / (pms / 1e3) / 1e9
    result = {
        "metric": "quicksort keys/s (uint64, n=2^%d, %s)" % (args.log2n, args.input),
        "value": value, "unit": "Gkeys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (SplitMix64 uniform keys, seeded; sorted / reverse / mod 16 "
                "derived from them)",
        "config": {"workload": "quicksort u64 n=2^%d input=%s" % (args.log2n, args.input),
                   "pivot": "median of %d seeded keys per subarray" % args.pivot_samples,
                   "n": n, "input": args.input,
                   "l2": "2 GiB input, regenerated on device between steps",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "batched_kernel<uint64_t> (every partition level, "
                               "with its set-up launches)",
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_step": 2 * 8 * pk, "ms_per_step": pms,
                     "sort_kernel": {"achieved": 2 * 8 * sk / (sms / 1e3) / 1e9 if sms else None,
                                     "ms_per_step": sms, "keys": sk}},
        "levels": stats[-1]["levels"],
        "partition_keys_per_key": pk / n,
        "gpu_launches": launches,
        "sorted_last_step": sorted_ok,
        "aux_bytes": ctx.aux_bytes,
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk
    if not args.no_e2e:
        host_in = torch.empty(n, dtype=torch.int64, pin_memory=True)
        host_out = torch.empty(n, dtype=torch.int64, pin_memory=True)
        fill_sort_input(lp, keys, args.input, seed0 + 555)
        host_in.copy_(keys)
        torch.cuda.synchronize()
        times = []
        for k in range(max(1, args.e2e_steps)):
            ev0.record(stream)
            keys.copy_(host_in, non_blocking=True)
            lp.lp_quicksort(ctx, keys, seed=k, pivot_samples=args.pivot_samples)
            host_out.copy_(keys, non_blocking=True)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
        keys_all, e_ms = whole_job(ws, n, sum(times) / len(times))
        result["e2e"] = {"value": keys_all / (e_ms / 1e3) / 1e9, "unit": "Gkeys/s",
                         "ms_per_step": e_ms,
                         "h2d_bytes_per_step": 8 * n * ws, "d2h_bytes_per_step": 8 * n * ws,
                         "path": "pinned host -> device, lp_quicksort_u64, device -> pinned host"}
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, ns, reps, med = cpu_oracle_sort(args.input, min(args.log2n, 22), args.seed)
        result["cpu_baseline"] = {
            "value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "2^%d uint64 keys, same input kind, median of %d runs (%.2f s each) of "
                      "the serial quicksort" % (int(np.log2(ns)), reps, med),
            "host_cores_available": os.cpu_count()}
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- batched

def batch_layout(count, seed):
    """Sizes log-uniform in [2^8, 2^22] and 16-byte aligned offsets in one buffer."""
    sizes = inputs.log_uniform_sizes(count, seed, 8, 22)
    offs, tot = [], 0
    for m in sizes:
        offs.append(tot)
        tot += (int(m) + 1) & ~1
    return sizes, offs, tot


def cpu_oracle_batch(sizes, seed, budget_s):
    """The serial oracle over the batch's instances in order, for about budget_s
    seconds of partition time; returns (Gkeys/s, keys, instances)."""
    import oracle
    rng = np.random.default_rng(seed)
    spent, done, inst = 0.0, 0, 0
    for s, m in enumerate(sizes):
        a = inputs.uniform_u64(int(m), seed + s)
        p = int(a[int(rng.integers(0, m))])
        t0 = time.perf_counter()
        oracle.partition(a, p)
        spent += time.perf_counter() - t0
        done += int(m)
        inst += 1
        if spent > budget_s:
            break
    return done / spent / 1e9, done, inst


def run_batched(args):
    import torch
    ws, rank, local = dist_env()
    init_dist(local, ws)
    from paper_2004_12532_gb300 import binding as lp
    count = args.instances
    sizes, offs, tot = batch_layout(count, args.seed)
    keys_total = int(sum(int(m) for m in sizes))
    buf = torch.empty(tot, dtype=torch.int64, device="cuda")
    seed0 = args.seed + 7919 * rank
    # every step partitions the same seeded input (regenerated on the device,
    # 14 GB > L2), so each pivot stays a seeded random element of its segment
    lp.lp_fill_uniform_u64(buf, seed0)
    rng = np.random.default_rng(args.seed)
    pick = [o + int(rng.integers(0, m)) for o, m in zip(offs, sizes)]
    pv = buf[torch.tensor(pick, dtype=torch.int64, device="cuda")].cpu().numpy()
    pivots = [int(x) & 0xFFFFFFFFFFFFFFFF for x in pv]
    views = [buf[o:o + int(m)] for o, m in zip(offs, sizes)]
    splits = torch.zeros(count, dtype=torch.int64, device="cuda")
    splits_plain = torch.zeros(count, dtype=torch.int64, device="cuda")
    ctx = lp.Ctx(local)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tuning = lp.lp_autotune_batched_u64(ctx, [int(m) for m in sizes])
    tune_s = time.perf_counter() - t0
    batch = lp.Batch(ctx, views, pivots, splits, seed=1)
    for w in range(args.warmup):
        lp.lp_fill_uniform_u64(buf, seed0)
        batch.launch()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    g_ms, streamed, launches = [], [], 0
    wall0 = time.perf_counter()
    clocks.start()
    for k in range(args.steps):
        lp.lp_fill_uniform_u64(buf, seed0)
        ev0.record(stream)
        batch.launch()
        ev1.record(stream)
        ev1.synchronize()
        g_ms.append(ev0.elapsed_time(ev1))
        launches += ctx.last_launches
        streamed.append(batch.streamed_keys())
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - wall0
    clk = clocks.stop()
    # the same instances as separate plain launches (lp_partition_u64_async each)
    p_ms, p_launches = [], 0
    for k in range(max(1, min(args.steps, 3))):
        lp.lp_fill_uniform_u64(buf, seed0)
        torch.cuda.synchronize()
        ev0.record(stream)
        for s in range(count):
            lp.lp_partition_u64_async(ctx, views[s], pivots[s], splits_plain[s:s + 1], seed=k)
            p_launches += ctx.last_launches
        ev1.record(stream)
        ev1.synchronize()
        p_ms.append(ev0.elapsed_time(ev1))
    same_splits = bool(torch.equal(splits, splits_plain))
    ms = sum(g_ms) / len(g_ms)
    keys_all, ms_all = whole_job(ws, keys_total, ms)
    value = keys_all / (ms_all / 1e3) / 1e9
    plain_ms = sum(p_ms) / len(p_ms)
    peak, peak_kind = measured_peaks()
    sk = sum(streamed) / len(streamed)
    achieved = 2 * 8 * sk / (ms / 1e3) / 1e9
    result = {
        "metric": "batched partition keys/s (%d uint64 instances, sizes log-uniform "
                  "[2^8, 2^22])" % count,
        "value": value, "unit": "Gkeys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (SplitMix64 uniform keys, seeded; pivot = seeded random element "
                "of each instance)",
        "config": {"workload": "batched partition, %d instances, %d keys in all" % (
                       count, keys_total),
                   "instances": count, "keys": keys_total, "tuning": tuning,
                   "autotune_s": tune_s,
                   "l2": "inputs larger than L2 (%.1f GB), regenerated on device between steps"
                         % (8 * keys_total / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "batched_kernel<uint64_t> (one graph: set-up kernel + "
                               "persistent kernel)",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": 2 * 8 * sk,
                     "ms_per_launch": ms},
        "per_instance_launches": {"value": keys_total / (plain_ms / 1e3) / 1e9,
                                  "unit": "Gkeys/s", "ms_per_step": plain_ms,
                                  "calls": count, "gpu_launches": p_launches // len(p_ms),
                                  "speedup_of_batched": plain_ms / ms,
                                  "same_splits": same_splits},
        "streamed_keys_per_key": sk / keys_total,
        "gpu_launches": launches,
        "aux_bytes": ctx.aux_bytes,
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk
    if not args.no_e2e:
        host_in = torch.empty(tot, dtype=torch.int64, pin_memory=True)
        host_out = torch.empty(tot, dtype=torch.int64, pin_memory=True)
        host_splits = torch.empty(count, dtype=torch.int64, pin_memory=True)
        lp.lp_fill_uniform_u64(buf, seed0)
        host_in.copy_(buf)
        torch.cuda.synchronize()
        times = []
        for k in range(max(1, args.e2e_steps)):
            ev0.record(stream)
            buf.copy_(host_in, non_blocking=True)
            batch.launch()
            host_out.copy_(buf, non_blocking=True)
            host_splits.copy_(splits, non_blocking=True)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
        keys_all, e_ms = whole_job(ws, keys_total, sum(times) / len(times))
        result["e2e"] = {"value": keys_all / (e_ms / 1e3) / 1e9, "unit": "Gkeys/s",
                         "ms_per_step": e_ms, "h2d_bytes_per_step": 8 * tot * ws,
                         "d2h_bytes_per_step": (8 * tot + 8 * count) * ws,
                         "path": "pinned host -> device, graph launch of the batch, "
                                 "device -> pinned host (keys and splits)"}
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, done, inst = cpu_oracle_batch(sizes, args.seed, 10.0)
        result["cpu_baseline"] = {
            "value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d instances (%d keys), serial two-pointer partition, pivot "
                      "a seeded element of each" % (inst, done),
            "host_cores_available": os.cpu_count()}
    batch.close()
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- serve

def serve_requests(lp, count, rate, seed):
    """Poisson arrivals (mean `rate` per s), 70% partition / 30% sort, sizes
    log-uniform in [2^10, 2^26], uint32 or uint64 keys with equal probability,
    uniform keys generated on the device from each request's seed; a
    partition's pivot is the key value at a seeded quantile in [1%, 99%]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    t -= t[0]
    sizes = inputs.log_uniform_sizes(count, seed, 10, 26)
    reqs = []
    for i in range(count):
        kind = lp.LP_REQ_SORT if rng.random() < 0.3 else lp.LP_REQ_PARTITION
        bits = 64 if rng.random() < 0.5 else 32
        pivot = inputs.quantile_pivot(int(rng.integers(1, 100)), 100, bits)
        reqs.append(lp.Server.request(kind, bits, int(sizes[i]), pivot,
                                      (seed << 20) + i, None, float(t[i])))
    return reqs


def latency_summary(reqs, out):
    lat = np.array([c["done_s"] - c["arrival_s"] for c in out]) * 1e3
    keys = sum(r.n for r in reqs)
    span = max(c["done_s"] for c in out) - min(c["arrival_s"] for c in out)
    part = [l for r, l in zip(reqs, lat) if r.kind == 0]
    sort = [l for r, l in zip(reqs, lat) if r.kind == 1]
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "p50_partition_ms": float(np.percentile(part, 50)) if part else None,
            "p99_partition_ms": float(np.percentile(part, 99)) if part else None,
            "p50_sort_ms": float(np.percentile(sort, 50)) if sort else None,
            "p99_sort_ms": float(np.percentile(sort, 99)) if sort else None,
            "keys": keys, "span_s": span, "gkeys_per_s": keys / span / 1e9}


def run_serve(args):
    import torch
    ws, rank, local = dist_env()
    init_dist(local, ws)
    from paper_2004_12532_gb300 import binding as lp
    budget = int(args.budget_gib * (1 << 30))
    srv = lp.Server(local, budget_bytes=budget, max_slots=args.slots, seed=args.seed,
                    timing=True)
    seed0 = args.seed + 7919 * rank
    for w in range(args.warmup):
        srv.run(serve_requests(lp, max(50, args.requests // 10), args.rate, seed0 + 900 + w))
    st0 = srv.stats()
    s64_0, s32_0 = srv.streamed_keys()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    summaries, all_lat, keys_total, span_total = [], [], 0, 0.0
    wall0 = time.perf_counter()
    for k in range(args.steps):
        reqs = serve_requests(lp, args.requests, args.rate, seed0 + k)
        out = srv.run(reqs)
        summ = latency_summary(reqs, out)
        summaries.append(summ)
        all_lat += [(c["done_s"] - c["arrival_s"]) * 1e3 for c in out]
        keys_total += summ["keys"]
        span_total += summ["span_s"]
    wall_s = time.perf_counter() - wall0
    clk = clocks.stop()
    st1 = srv.stats()
    s64_1, s32_1 = srv.streamed_keys()
    # the first step's requests again, one at a time through the plain calls
    reqs0 = serve_requests(lp, args.requests, args.rate, seed0)
    base = latency_summary(reqs0, srv.run(reqs0, mode=lp.LP_SERVE_ONE_AT_A_TIME))
    ms = span_total / args.steps * 1e3
    keys_all, ms_all = whole_job(ws, keys_total / args.steps, ms)
    value = keys_all / (ms_all / 1e3) / 1e9
    lat = np.array(all_lat)
    peak, peak_kind = measured_peaks()
    b_ms = st1["batched_ms"] - st0["batched_ms"]
    b_bytes = 2 * (8 * (s64_1 - s64_0) + 4 * (s32_1 - s32_0))
    achieved = b_bytes / (b_ms / 1e3) / 1e9 if b_ms > 0 else None
    result = {
        "metric": "served keys/s (Poisson %.0f req/s, 70%% partition / 30%% sort, sizes "
                  "log-uniform [2^10, 2^26], uint32/uint64)" % args.rate,
        "value": value, "unit": "Gkeys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64",
        "data": "synthetic (seeded Poisson arrivals; uniform keys generated on the device "
                "from each request's seed on admission)",
        "config": {"workload": "serve %d requests per step at %.0f req/s" % (
                       args.requests, args.rate),
                   "budget_gib": args.budget_gib, "slots": args.slots,
                   "requests_per_step": args.requests,
                   "l2": "request keys regenerated on admission; working set above L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "latency": {"p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)),
                    "per_step": summaries},
        "one_at_a_time": base,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "batched_kernel (uint64 and uint32 launches of the engine "
                               "steps)", "peak_kind": peak_kind,
                     "algorithmic_bytes": b_bytes, "ms": b_ms},
        "engine": {"steps": st1["steps"] - st0["steps"],
                   "launches": st1["launches"] - st0["launches"],
                   "peak_bytes": st1["peak_bytes"], "engine_bytes": st1["engine_bytes"],
                   "busy_s": st1["busy_s"] - st0["busy_s"]},
        "gpu_launches": st1["launches"] - st0["launches"],
        "e2e": None,
        "e2e_note": "requests' keys are device-resident by design (generated on admission)",
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk
    srv.close()
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.log2n is None:
        args.log2n = 28 if args.workload == "quicksort" else \
            {"u64": 30, "u32": 31, "kv": 29}[args.dtype]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "quicksort":
        run_quicksort(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
