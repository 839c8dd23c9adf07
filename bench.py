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
HANDOFF = (1 << 64) - 1  # level record of a range handed to the low-space partition
# The kernel sources each committed ncu summary (profiles/) was taken on; a
# summary feeds roofline.traffic only while the hash of these files matches.
PART_SOURCES = ["lp_smoothed.cuh", "lp_kernels.cu", "lp_plan.h", "lp_device.cuh",
                "lp_coop.cuh", "lp_launch.h"]
BATCH_SOURCES = ["lp_batched.cu", "lp_batched.h", "lp_batch_init.cuh", "lp_smoothed.cuh",
                 "lp_plan.h", "lp_device.cuh", "lp_coop.cuh", "lp_fixup.cuh"]
QS_SOURCES = BATCH_SOURCES + ["lp_qs.cu", "lp_qs.cuh", "lp_qs_sort.cuh", "lp_qs_pivot.cuh",
                              "lp_qs_level.cuh", "lp_qs_local.cu", "lp_quicksort.cu"]
# name -> (summary file, kernel sources, machine-readable key of its DRAM bytes per unit)
PROFILES = {
    "partition_u64": ("partition_kernel_ncu.txt", PART_SOURCES, "dram_bytes_per_key"),
    "partition_u32": ("partition_kernel_ncu.txt", PART_SOURCES, "dram_bytes_per_key_u32"),
    "partition_kv": ("partition_kernel_ncu.txt", PART_SOURCES, "dram_bytes_per_key_kv"),
    "batched": ("batched_kernel_u64_ncu.txt", BATCH_SOURCES, "dram_bytes_per_streamed_key"),
    "quicksort": ("quicksort_u64_2p28_ncu.txt", QS_SOURCES, "dram_bytes_per_streamed_key"),
}


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
    ap.add_argument("--no-subs", action="store_true",
                    help="default run: skip the other workloads' objects (u32, key+payload, "
                         "quicksort, batched, serve)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_hash(sources=None):
    """Hash of kernel sources without // comments and blank lines (a comment
    changes no kernel)."""
    h = hashlib.sha256()
    for f in (sources or PART_SOURCES):
        for line in open(os.path.join(ROOT, "paper_2004_12532_gb300", "csrc", f), "rb"):
            code = line.split(b"//", 1)[0].rstrip()
            if code:
                h.update(code + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(name, units):
    """(DRAM read + write bytes per launch, None) from the committed ncu summary
    `name`, scaled to `units` (keys of the launch), if that summary was taken on
    the current kernel sources; else (None, why not)."""
    fname, sources, key = PROFILES[name]
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None, "no ncu summary committed"
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith(" "):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_hash(sources):
        return None, "the kernel changed since its ncu capture"
    try:
        per_unit = float(kv[key])
    except (KeyError, ValueError):
        return None, "the ncu summary has no %s" % key
    return per_unit * units, None


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


def cpu_oracle_partition(dt, log2n, pivot, seed, min_seconds):
    """cpu_baseline of a partition workload: the serial oracle (two-pointer
    partition; with payloads, key and payload swapped together) on a bounded
    sample of the same distribution and pivot, one host core."""
    import oracle
    ls = min(log2n, 27 if dt == "u64" else 26)
    n = 1 << ls
    times = []
    t_start = time.time()
    for r in range(5):
        a = inputs.uniform_u32(n, seed + r) if dt == "u32" else inputs.uniform_u64(n, seed + r)
        v = np.arange(n, dtype=np.uint64) if dt == "kv" else None
        t0 = time.perf_counter()
        if v is None:
            oracle.partition(a, pivot)
        else:
            oracle.partition_kv(a, v, pivot)
        times.append(time.perf_counter() - t0)
        if time.time() - t_start > min_seconds and len(times) >= 2:
            break
    med = statistics.median(times)
    E = {"u64": 8, "u32": 4, "kv": 16}[dt]
    what = {"u64": "uint64 keys", "u32": "uint32 keys",
            "kv": "uint64 key + uint64 payload pairs"}[dt]
    return {"value": 3 * E * n / med / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "2^%d %s, same distribution and pivot, median of %d runs (%.2f s each) "
                      "of the serial two-pointer partition" % (ls, what, len(times), med),
            "host_cores_available": os.cpu_count()}


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
    n = 1 << args.log2n
    # the full workload: one input generated once, restored before each timed
    # step (untimed); warm-up steps on a 2^24-key slice of it
    master = inputs.uniform_u64(n, args.seed)
    work = np.empty_like(master)
    for w in range(args.warmup):
        a = master[:1 << min(24, args.log2n)].copy()
        oracle.partition(a, pivot)
    total = 0.0
    for k in range(args.steps):
        np.copyto(work, master)
        t0 = time.perf_counter()
        oracle.partition(work, pivot)
        total += time.perf_counter() - t0
    ms = total / args.steps * 1e3
    value = 3 * 8 * n / (ms / 1e3) / 1e9
    sample = ("the whole workload: 2^%d uint64 keys per step, same distribution and pivot "
              "(one seeded input, restored before each step)" % args.log2n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": partition_config(args, "u64", args.log2n, n, pivot, 1),
        "reference": "the oracle: serial two-pointer partition (CPU), one host core",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def partition_config(args, dt, log2n, n, pivot, ws):
    """The config object of a partition workload (both arms print the same)."""
    return {"workload": "partition %s n=2^%d pivot at %d%% quantile, %s" % (
                dt, log2n, args.quantile, args.variant),
            "n": n, "pivot": pivot, "variant": args.variant, "dtype": dt,
            "l2": "inputs larger than L2 (8 GiB), regenerated on device between steps",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


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


# ---------------------------------------------------------------- parity
# In-run checks of a result against properties that hold at any size (the
# plain definition of the problem): the split equals the predicate count, the
# postcondition holds, and the array is a permutation of its input, the last
# by an order-independent fingerprint (two wrapping sums of a 64-bit mixer,
# Murmur3's finalizer, over every key).  Device-side torch ops, outside the
# timed regions.

def _s64(c):
    """A 64-bit constant as the int64 value with the same bits."""
    c &= (1 << 64) - 1
    return c - (1 << 64) if c >= (1 << 63) else c


_FM1, _FM2, _FALT = _s64(0xFF51AFD7ED558CCD), _s64(0xC4CEB9FE1A85EC53), _s64(0x9E3779B97F4A7C15)
_CHUNK = 1 << 27


def _bits64(x):
    """int32 -> int64 with the uint32 value; int64 unchanged."""
    import torch
    return (x.to(torch.int64) & 0xFFFFFFFF) if x.dtype == torch.int32 else x


def _fmix(x):
    m = (1 << 31) - 1  # logical shift by 33 on int64 bits
    x = x ^ ((x >> 33) & m)
    x = x * _FM1
    x = x ^ ((x >> 33) & m)
    x = x * _FM2
    return x ^ ((x >> 33) & m)


def fingerprint(keys, vals=None):
    """Order-independent fingerprint of a key array (or of its (key, value)
    pairs): equal for any permutation, different for any other multiset but
    with negligible probability."""
    a = b = 0
    for i in range(0, keys.numel(), _CHUNK):
        k = _bits64(keys[i:i + _CHUNK])
        if vals is not None:
            k = _fmix(k) ^ _fmix(vals[i:i + _CHUNK] ^ _FALT) * 3
        a = (a + int(_fmix(k).sum().item())) & ((1 << 64) - 1)
        b = (b + int(_fmix(k ^ _FALT).sum().item())) & ((1 << 64) - 1)
    return a, b


def count_le(keys, pivot):
    """Keys <= pivot, in the unsigned order of their bits."""
    c = 0
    if keys.dtype.itemsize == 4:
        for i in range(0, keys.numel(), _CHUNK):
            c += int((_bits64(keys[i:i + _CHUNK]) <= int(pivot)).sum().item())
        return c
    pv = _s64(int(pivot) ^ (1 << 63))
    for i in range(0, keys.numel(), _CHUNK):
        c += int(((keys[i:i + _CHUNK] ^ _s64(1 << 63)) <= pv).sum().item())
    return c


def partition_holds(keys, t, pivot):
    """keys[0..t) <= pivot < keys[t..n)."""
    return count_le(keys[:t], pivot) == t and count_le(keys[t:], pivot) == 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    init_dist(local, ws)
    from paper_2004_12532_gb300 import binding as lp
    result = measure_partition(args, lp, args.dtype, args.log2n, extras=True)
    if (args.dtype == "u64" and args.log2n == 30 and args.variant == "smoothed" and
            args.quantile == 50 and not args.no_subs):
        result.update(sub_results(args, lp))
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()


def sub_args(args):
    """The other workloads of the default run: at most 5 timed steps after at
    least 3 warm-up steps each, device-timed only (the headline carries e2e)."""
    import copy
    a = copy.copy(args)
    a.steps = max(1, min(args.steps, 5))
    a.warmup = max(3, min(args.warmup, 3))
    a.no_e2e = True
    a.no_yardstick = True
    return a


def sub_results(args, lp):
    """Every other workload in the default run, one object each: the partition
    of 2^31 uint32 keys and of 2^29 key + payload pairs, the quicksort of 2^28
    uint64 keys on its four inputs, the batched partition of 4096 instances and
    the serving run."""
    import torch
    sa = sub_args(args)
    out = {}
    torch.cuda.empty_cache()
    out["u32_2p31"] = measure_partition(sa, lp, "u32", 31)
    torch.cuda.empty_cache()
    out["kv_2p29"] = measure_partition(sa, lp, "kv", 29)
    torch.cuda.empty_cache()
    qs = {}
    for inp in ("uniform", "sorted", "reverse", "dup16"):
        qa = copy_with(sa, input=inp, log2n=28)
        qs[inp] = measure_quicksort(qa, lp)
        torch.cuda.empty_cache()
    out["quicksort_2p28"] = qs
    out["batched"] = measure_batched(copy_with(sa, instances=4096), lp)
    torch.cuda.empty_cache()
    out["serve"] = measure_serve(copy_with(sa, steps=min(sa.steps, 2), warmup=1,
                                           requests=1000, rate=2000.0), lp)
    torch.cuda.empty_cache()
    return out


def copy_with(args, **kw):
    import copy
    a = copy.copy(args)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def measure_partition(args, lp, dt, log2n, extras=False):
    """One partition workload: `dt` keys ("u64", "u32" or "kv": uint64 keys
    with uint64 payloads), n = 2^log2n, the pivot at args.quantile; returns its
    JSON object.  extras: the out-of-place yardstick, the e2e leg through the
    host-array entry point and the CPU baselines (u64 only)."""
    import torch
    ws, rank, local = dist_env()
    n = 1 << log2n
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
    levels_seen, level_ms, handoffs = [], [], 0
    pre = None
    barrier()
    wall0 = time.perf_counter()
    clocks.start()
    for k in range(args.steps):
        fill(seed0 + k)
        if k == args.steps - 1:  # the last step's input, for the parity checks (untimed)
            pre = (count_le(keys, pivot), fingerprint(keys, vals))
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
        # a range handed to the low-space partition is not streamed by this kernel
        traffic_keys.append(sum(hi - lo for lo, hi, _, g, _ in st if g != HANDOFF))
        handoffs += sum(1 for _, _, _, g, _ in st if g == HANDOFF)
        levels_seen.append([(hi - lo) for lo, hi, _, _, _ in st if hi > lo])
        level_ms.append([ms_ for _, _, _, _, ms_ in st])
    barrier()
    wall_s = time.perf_counter() - wall0
    clk = clocks.stop()
    t = int(d_split.item())
    parity = {"split_equals_count": t == pre[0],
              "postcondition": partition_holds(keys, t, pivot),
              "permutation_fingerprint": fingerprint(keys, vals) == pre[1],
              "checked": "last timed step: split vs the count of keys <= pivot, "
                         "keys[0..t) <= pivot < keys[t..n), multiset fingerprint of "
                         "the %s before and after" % ("(key, payload) pairs" if vals is not
                                                      None else "keys")}
    parity["ok"] = all(v for k_, v in parity.items() if k_ != "checked")

    ms = sum(part_ms) / len(part_ms)
    bytes_all, ms_all = whole_job(ws, 3 * E * n, ms)
    value = bytes_all / (ms_all / 1e3) / 1e9

    peak, peak_kind = measured_peaks()
    k_ms = sum(kern_ms) / len(kern_ms)
    k_keys = sum(traffic_keys) / len(traffic_keys)
    kname = {"u64": "uint64_t", "u32": "uint32_t", "kv": "uint64_t, payload"}[dt]
    basis = None
    traffic_note = None
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
        traffic_note = ("not scaled from a small capture: at 2^26 a quarter of the "
                        "MakeSuccessorHeavy traffic stays in L2, at full size almost none")
    else:
        k_bytes = 2 * E * k_keys  # one read and one write of every key of every level
        kernel = "partition_kernel<%s> (all levels, one cooperative launch)" % kname
        traffic, traffic_note = (profiled_traffic("partition_" + dt, k_keys)
                                 if args.variant == "smoothed"
                                 else (None, "no capture of this variant"))
    achieved = k_bytes / (k_ms / 1e3) / 1e9
    l0_ms = sum(lvl0_ms) / len(lvl0_ms)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": k_bytes,
                "ms_per_launch": k_ms,
                "level0_gbs_device_timestamps": 2 * E * (sum(lvl0_n) / len(lvl0_n)) /
                (l0_ms / 1e3) / 1e9 if l0_ms > 0 else None}
    if traffic is None and traffic_note:
        roofline["traffic_note"] = traffic_note
    if basis:
        roofline["basis"] = basis

    metric = METRIC if (dt == "u64" and log2n == 30) else \
        "in-place partition GB/s (%s, n=2^%d)" % ({"u64": "uint64", "u32": "uint32",
                                                   "kv": "uint64 key + uint64 payload"}[dt],
                                                  log2n)
    result = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if dt == "u32" else "u64",
        "data": "synthetic (SplitMix64 uniform keys, seeded)",
        "config": partition_config(args, dt, log2n, n, pivot, ws),
        "roofline": roofline,
        "gpu_launches": launches,
        "parity": parity,
        "split_last_step": t,
        # physical read + write bytes of the partition kernel's levels over the step time
        "true_gbs": ws * 2 * E * k_keys / (ms_all / 1e3) / 1e9,
        "level_ranges_last_step": levels_seen[-1],
        "level_ms_mean": [round(sum(x) / len(x), 4) for x in zip(*level_ms)],
        "handoffs": handoffs,
        "aux_bytes": ctx.aux_bytes,
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk

    if extras and not args.no_yardstick and dt == "u64":
        result["yardstick_cub"] = cub_yardstick(args, keys, n, pivot, stream, fill, seed0, t)
        result["yardstick_standard"] = standard_yardstick(args, keys, n, pivot, stream, fill,
                                                          seed0, t)
    if extras and not args.no_e2e and dt == "u64" and args.variant == "smoothed":
        result["e2e"] = e2e_leg(args, lp, ctx, keys, d_split, pivot, variant, n, seed0, stream)
    if rank == 0 and ws == 1 and not args.no_cpu:
        if extras and dt == "u64":
            result["cpu_parallel"] = cpu_parallel_gbs(min(log2n, 27), pivot, args.seed)
        result["cpu_baseline"] = cpu_oracle_partition(dt, log2n, pivot, args.seed,
                                                      8.0 if extras else 4.0)
    ctx.close()
    return result


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


def standard_yardstick(args, keys, n, pivot, stream, fill, seed0, split_ours):
    """The paper's Standard linear-space partition (Sec. 2: prefix sums S in an
    array of n counts, reorder into C, copy back; libyardstick.so) of the same
    input, timed the same way: the high-space baseline of the paper's
    experiments, on this GPU.  Not the product path."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_2004_12532_gb300", "libyardstick.so")
    if not os.path.exists(path):
        return {"unavailable": "libyardstick.so not built"}
    L = ctypes.CDLL(path)
    L.yd_standard_scratch_words.restype = ctypes.c_uint64
    L.yd_standard_scratch_words.argtypes = [ctypes.c_uint64]
    L.yd_standard_partition_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    words = L.yd_standard_scratch_words(n)
    scratch = torch.empty(words, dtype=torch.int64, device="cuda")
    sel = torch.zeros(1, dtype=torch.int64, device="cuda")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    for k in range(max(3, args.warmup) + max(3, min(args.steps, 5))):
        fill(seed0 + k)
        ev0.record(stream)
        rc = L.yd_standard_partition_u64(keys.data_ptr(), n, pivot, scratch.data_ptr(),
                                         sel.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        ev1.synchronize()
        if rc != 0:
            return {"unavailable": "standard partition failed"}
        if k >= max(3, args.warmup):
            times.append(ev0.elapsed_time(ev1))
    fill(seed0 + args.steps - 1)  # the last timed input of our partition, for the split
    L.yd_standard_partition_u64(keys.data_ptr(), n, pivot, scratch.data_ptr(), sel.data_ptr(),
                                stream.cuda_stream)
    torch.cuda.synchronize()
    ms = sum(times) / len(times)
    res = {"kernel": "Standard linear-space partition (Sec. 2; prefix phase, reorder into C, "
                     "copy back)", "ms_per_step": ms,
           "effective_gbs": 3 * 8 * n / (ms / 1e3) / 1e9,
           # algorithmic traffic: count pass (8n), prefix pass (read 8n, write S 8n),
           # reorder (read A and S, write C: 24n), copy back (16n)
           "algorithmic_gbs": 64 * n / (ms / 1e3) / 1e9,
           "extra_device_bytes": 8 * words,
           "same_split": int(sel.item()) == split_ours}
    del scratch
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
    result = measure_quicksort(args, lp)
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()


def measure_quicksort(args, lp):
    """The quicksort workload (n = 2^args.log2n uint64 keys, input args.input);
    returns its JSON object."""
    import torch
    ws, rank, local = dist_env()
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
    pre = None
    wall0 = time.perf_counter()
    clocks.start()
    for k in range(args.steps):
        fill_sort_input(lp, keys, args.input, seed0 + k)  # untimed; 2 GiB > L2
        if k == args.steps - 1:
            pre = fingerprint(keys)
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
    parity = {"sorted": sorted_ok, "permutation_fingerprint": fingerprint(keys) == pre,
              "checked": "last timed step: every key <= the next (unsigned), multiset "
                         "fingerprint of the keys before and after (the sorted output is "
                         "unique, so these fix it)"}
    parity["ok"] = parity["sorted"] and parity["permutation_fingerprint"]
    ms = sum(step_ms) / len(step_ms)
    keys_all, ms_all = whole_job(ws, n, ms)
    value = keys_all / (ms_all / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    pk = sum(s_["partition_keys"] for s_ in stats) / len(stats)
    pms = sum(s_["partition_ms"] for s_ in stats) / len(stats)
    sk = sum(s_["sort_keys"] for s_ in stats) / len(stats)
    sms = sum(s_["sort_ms"] for s_ in stats) / len(stats)
    tk = sum(s_["tail_keys"] for s_ in stats) / len(stats)
    tms = sum(s_["tail_ms"] for s_ in stats) / len(stats)
    achieved = 2 * 8 * pk / (pms / 1e3) / 1e9
    traffic, why = None, ("the committed ncu summary (profiles/quicksort_u64_2p28_ncu.txt) "
                          "captures single levels; a step's traffic is not one level's scaled")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "batched_kernel<uint64_t> (every partition level, "
                          "with its set-up launches)",
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_step": 2 * 8 * pk, "ms_per_step": pms,
                "sort_kernel": {"achieved": 2 * 8 * sk / (sms / 1e3) / 1e9 if sms else None,
                                "ms_per_step": sms, "keys": sk},
                "tail_kernel": {"ms_per_step": tms, "streamed_keys": tk,
                                "items": stats[-1]["tail_items"]},
                # the whole sort: every key streamed by a partition (levels and tail)
                # or sorted on chip is read and written once (2K bytes), over the
                # step time
                "whole_sort": {"algorithmic_bytes": 2 * 8 * (pk + tk + sk), "ms": ms,
                               "achieved": 2 * 8 * (pk + tk + sk) / (ms / 1e3) / 1e9,
                               "frac": 2 * 8 * (pk + tk + sk) / (ms / 1e3) / 1e9 / peak}}
    if traffic is None:
        roofline["traffic_note"] = why
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
        "roofline": roofline,
        "levels": stats[-1]["levels"],
        "partition_keys_per_key": (pk + tk) / n,
        "gpu_launches": launches,
        "parity": parity,
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
        v, ns, reps, med = cpu_oracle_sort(args.input, min(args.log2n, 22), args.seed,
                                           min_seconds=2.0 if args.steps <= 5 else 8.0)
        result["cpu_baseline"] = {
            "value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "2^%d uint64 keys, same input kind, median of %d runs (%.2f s each) of "
                      "the serial quicksort" % (int(np.log2(ns)), reps, med),
            "host_cores_available": os.cpu_count()}
    ctx.close()
    return result


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
    result = measure_batched(args, lp)
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()


def segment_fingerprints(buf, offs, sizes):
    """One wrapping 64-bit sum of the mixed keys per segment (an
    order-independent fingerprint of each segment's multiset), from a prefix
    sum over the whole buffer."""
    import torch
    F = torch.empty_like(buf)
    for i in range(0, buf.numel(), _CHUNK):
        F[i:i + _CHUNK] = _fmix(buf[i:i + _CHUNK])
    F.cumsum_(0)
    ends = torch.tensor([o + int(m) - 1 for o, m in zip(offs, sizes)], device=buf.device)
    starts = torch.tensor([o - 1 for o in offs], device=buf.device)
    before = torch.where(starts >= 0, F[starts.clamp(min=0)], torch.zeros_like(starts))
    out = (F[ends] - before).cpu().tolist()
    del F
    return out


def measure_batched(args, lp):
    """The batched workload (args.instances uint64 instances, sizes log-uniform in
    [2^8, 2^22]) against the same instances as plain launches; returns its JSON
    object."""
    import torch
    ws, rank, local = dist_env()
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
    lp.lp_fill_uniform_u64(buf, seed0)
    pre_fp = segment_fingerprints(buf, offs, sizes)  # every step's input (untimed)
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
    # parity of the last timed launch's result, segment by segment
    got = splits.cpu().tolist()
    seg_ok = all(partition_holds(views[s_], got[s_], pivots[s_]) for s_ in range(count))
    post_fp = segment_fingerprints(buf, offs, sizes)
    lp.lp_fill_uniform_u64(buf, seed0)
    counts_ok = all(count_le(views[s_], pivots[s_]) == got[s_] for s_ in range(count))
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
    parity = {"splits_equal_counts": counts_ok, "postcondition_every_segment": seg_ok,
              "permutation_fingerprint_every_segment": pre_fp == post_fp,
              "same_splits_as_plain_launches": same_splits,
              "checked": "last timed launch: each segment's split vs the count of its keys "
                         "<= its pivot, the postcondition in each segment, each segment's "
                         "multiset fingerprint before and after; splits of the %d plain "
                         "launches" % count}
    parity["ok"] = counts_ok and seg_ok and pre_fp == post_fp and same_splits
    ms = sum(g_ms) / len(g_ms)
    keys_all, ms_all = whole_job(ws, keys_total, ms)
    value = keys_all / (ms_all / 1e3) / 1e9
    plain_ms = sum(p_ms) / len(p_ms)
    peak, peak_kind = measured_peaks()
    sk = sum(streamed) / len(streamed)
    achieved = 2 * 8 * sk / (ms / 1e3) / 1e9
    traffic, traffic_why = profiled_traffic("batched", sk)
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
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "batched_kernel<uint64_t> (one graph: set-up kernel + "
                               "persistent kernel)",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": 2 * 8 * sk,
                     "ms_per_launch": ms},
        "per_instance_launches": {"value": keys_total / (plain_ms / 1e3) / 1e9,
                                  "unit": "Gkeys/s", "ms_per_step": plain_ms,
                                  "calls": count, "gpu_launches": p_launches // len(p_ms),
                                  "speedup_of_batched": plain_ms / ms,
                                  "same_splits": same_splits},
        "parity": parity,
        "streamed_keys_per_key": sk / keys_total,
        "gpu_launches": launches,
        "aux_bytes": ctx.aux_bytes,
        "wall_s_timed_region": wall_s,
    }
    if clk:
        result["clocks"] = clk
    if traffic is None:
        result["roofline"]["traffic_note"] = traffic_why
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
        v, done, inst = cpu_oracle_batch(sizes, args.seed, 3.0 if args.steps <= 5 else 10.0)
        result["cpu_baseline"] = {
            "value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d instances (%d keys), serial two-pointer partition, pivot "
                      "a seeded element of each" % (inst, done),
            "host_cores_available": os.cpu_count()}
    batch.close()
    ctx.close()
    return result


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
    result = measure_serve(args, lp)
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()


def serve_parity(lp, reqs, cont, one, sample_every=7):
    """Partition requests: the split of the continuous run equals that of the
    same requests one at a time, and for every sample_every-th partition request
    it equals the count of keys <= pivot of that request's keys, regenerated
    from its seed as the server generates them (lp_fill_uniform_*)."""
    import torch
    same, counted, ok_count = True, 0, True
    parts = [i for i, r in enumerate(reqs) if r.kind == lp.LP_REQ_PARTITION]
    for j, i in enumerate(parts):
        same = same and cont[i]["split"] == one[i]["split"]
        if j % sample_every == 0:
            r = reqs[i]
            kd = torch.empty(r.n, dtype=torch.int64 if r.key_bits == 64 else torch.int32,
                             device="cuda")
            (lp.lp_fill_uniform_u64 if r.key_bits == 64 else lp.lp_fill_uniform_u32)(kd, r.seed)
            ok_count = ok_count and count_le(kd, r.pivot) == cont[i]["split"]
            counted += 1
            del kd
    return {"partition_splits_same_in_both_modes": same, "splits_equal_counts": ok_count,
            "ok": same and ok_count,
            "checked": "the first step's %d partition requests: continuous vs one at a time; "
                       "%d of them against the count of their regenerated keys; sort "
                       "results are checked by the test suite (alone and in a mix)" % (
                           len(parts), counted)}


def measure_serve(args, lp):
    """The serving workload (Poisson arrivals at args.rate, args.requests per
    step) against the same requests one at a time; returns its JSON object."""
    import torch
    ws, rank, local = dist_env()
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
        if k == 0:
            first_out = out
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
    one = srv.run(reqs0, mode=lp.LP_SERVE_ONE_AT_A_TIME)
    base = latency_summary(reqs0, one)
    parity = serve_parity(lp, reqs0, first_out, one)
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
        "parity": parity,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "traffic_note": "mixed key widths and launch sizes; the batched "
                                     "kernel's capture (batched object) covers the kernel",
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
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, keys, served = cpu_oracle_serve(args.seed, 2.0 if args.steps <= 5 else 5.0)
        result["cpu_baseline"] = {
            "value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": "%d requests of the same mix in stream order (%d keys), one at a time: "
                      "serial two-pointer partition / serial quicksort, service time only"
                      % (served, keys),
            "host_cores_available": os.cpu_count()}
    srv.close()
    return result


def cpu_oracle_serve(seed, budget_s):
    """The oracle serving the request mix one request at a time on one host
    core, for about budget_s seconds of service time; (Gkeys/s, keys, requests)."""
    import oracle
    rng = np.random.default_rng(seed)
    sizes = inputs.log_uniform_sizes(4096, seed, 10, 26)
    spent, keys, served = 0.0, 0, 0
    for i, m in enumerate(sizes):
        if spent > budget_s:
            break
        bits = 64 if rng.random() < 0.5 else 32
        a = inputs.uniform_u64(int(m), seed + i) if bits == 64 else \
            inputs.uniform_u32(int(m), seed + i)
        sort = rng.random() < 0.3
        pivot = inputs.quantile_pivot(int(rng.integers(1, 100)), 100, bits)
        t0 = time.perf_counter()
        if sort:
            oracle.quicksort(a, i)
        else:
            oracle.partition(a, pivot)
        spent += time.perf_counter() - t0
        keys += int(m)
        served += 1
    return keys / spent / 1e9, keys, served


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
