#!/usr/bin/env python
"""Throughput of libbinar on GB300: GKeys/s and fraction of the HBM roofline.

Workload (one step = one complete in-place stable sort): 256M uint32 keys with
uint32 payloads equal to the original index, keys uniform over [0, 2^32)
(PCG64, seed 8113448 + 200), synthetic.  The input (2 GiB, larger than the
129 MB L2) is restored from a pristine device copy before every step; only the
sort is timed, with CUDA events on the sort's stream.

Prints one JSON line (rank 0).  Run as ``python bench.py [--gpus N --steps K
--warmup W]``; for N > 1 under torchrun every rank sorts its own replica
(no data exchange) and rank 0 reports the max-over-ranks time.
``--impl reference`` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GKeys/s and % HBM roofline (u32/u64, 1M–1G keys); serving p50/p99 ms"
UNIT = "GKeys/s"
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = "256M uint32 keys + uint32 index payload, uniform, stable in-place sort"


def workload_name(n: int, key: str, dist: str) -> str:
    kname = "uint64" if key == "u64" else "uint32"
    return f"{n >> 20}M {kname} keys + uint32 index payload, {dist}, stable in-place sort"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["binar", "reference"], default="binar")
    ap.add_argument("--n", type=int, default=0,
                    help="keys (default: 256M for uint32 keys, 128M for uint64 keys)")
    ap.add_argument("--key", choices=["u32", "u64"], default="u32",
                    help="pairs workload key type (payload: uint32 original index)")
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--workload", choices=["pairs", "segments", "serve", "inplace"], default="pairs",
                    help="pairs: 256M uint32+uint32 sort (the headline); segments: 20,000 "
                         "segments in one CUDA-graph launch vs one call per segment; serve: "
                         "the continuous-batching request loop vs one request per launch; "
                         "inplace: the same pairs sorted by the unstable in-place mode")
    ap.add_argument("--seg-len", type=int, default=0,
                    help="segments: equal segments of this many keys instead of the "
                         "20,000 log-uniform ones")
    ap.add_argument("--seg-prefix-bits", type=int, default=0,
                    help="segments: the keys of a segment share their top B bits, like the "
                         "jobs a full sort hands its finisher after B / 8 levels")
    ap.add_argument("--no-plain", action="store_true",
                    help="segments: skip the one-call-per-segment comparison")
    ap.add_argument("--no-autotune", action="store_true",
                    help="segments: library defaults instead of the autotuned configuration")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="serve: device-memory budget")
    ap.add_argument("--span-log2", type=int, default=16,
                    help="serve: request sizes floor(2^(10 + span U)) keys (16: 1K..64M)")
    ap.add_argument("--slots", type=int, default=4, help="serve: batches in flight")
    ap.add_argument("--linger-us", type=float, default=0.0,
                    help="serve: a small batch waits up to this long for more requests "
                         "of its class while other batches run")
    ap.add_argument("--plain-slots", type=int, default=0,
                    help="serve: stream slots of the one-request-per-launch form (0: --slots)")
    args = ap.parse_args()
    if args.n <= 0:
        args.n = (128 << 20) if (args.key == "u64" and args.workload == "pairs") else (256 << 20)
    return args


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# the files that hold the partition and finisher kernels and their helpers
KERNEL_FILES = ("binar_internal.cuh", "kernels.cuh")


def kernel_source_hash():
    """Hash of the code of the files that hold the timed kernels: comments and
    whitespace are dropped, so that a comment edit does not mark recorded
    counters as stale, and code elsewhere in the library does not count."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0811_3448_gb300", "csrc")
    for name in KERNEL_FILES:
        with open(os.path.join(csrc, name)) as f:
            code = f.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(name.encode())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, key_bytes: int, val_bytes: int, n: int):
    """DRAM bytes per launch of `kernel` on n records of this key / payload
    width, from the committed ncu summary: its per-record traffic (taken on a
    smaller case of the same widths) times n.  None if the kernels have changed
    since it was taken or it holds no capture of these widths."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    ent = d.get("kernels", {}).get(kernel)
    if ent is None or ent.get("key_bytes") != key_bytes or ent.get("val_bytes") != val_bytes:
        return None
    per_key = (ent["dram_bytes_read"] + ent["dram_bytes_write"]) / ent["measured_keys"]
    return int(round(per_key * n))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def cpu_baseline(n_sample: int, dist: str, kdt=np.uint32):
    """The oracle's parallel binar sort on the host cores, on a bounded sample."""
    import oracle
    from paper_0811_3448_gb300 import inputs
    cores = os.cpu_count() or 1
    log2g = max(0, int(math.floor(math.log2(cores))))
    keys = inputs.config2_keys(n_sample, kdt, dist)
    vals = inputs.index_payload(n_sample)
    k = keys.copy()
    t0 = time.perf_counter()
    oracle.binar_sort_parallel(k, vals, log2_groups=log2g)
    dt = time.perf_counter() - t0
    out = {"value": n_sample / dt / 1e9, "unit": UNIT, "cores": 1 << log2g, "kind": "oracle",
           "sample": f"{n_sample} {np.dtype(kdt).name} keys + uint32 payload ({dist}), parallel binar sort "
                     f"(leading-bit split, one thread per group), {dt:.2f} s wall",
           "validated": host_sorted_pairs(keys, k, vals)}
    # context, one host thread on a smaller sample: the paper's sequential
    # binar sort (keys alone, in place) and the library sort of numpy
    m = max(1, n_sample // 8)
    k1 = keys[:m].copy()
    t0 = time.perf_counter()
    oracle.binar_sort(k1)
    t1 = time.perf_counter()
    k2 = np.sort(keys[:m], kind="stable")
    t2 = time.perf_counter()
    out["single_thread"] = {
        "sample": f"{m} {np.dtype(kdt).name} keys ({dist}), keys alone",
        "binar_sort_GKeys_per_s": m / (t1 - t0) / 1e9,
        "numpy_sort_GKeys_per_s": m / (t2 - t1) / 1e9,
        "validated": bool(np.array_equal(k1, k2))}
    return out


def host_sorted_pairs(orig: np.ndarray, keys: np.ndarray, vals: np.ndarray) -> bool:
    """A CPU sort's output is nondecreasing and every payload (the original
    index) points at the key it travels with, each index once."""
    ok = bool(np.all(keys[1:] >= keys[:-1]))
    idx = vals.astype(np.int64)
    ok &= bool(np.array_equal(np.sort(idx), np.arange(len(orig), dtype=np.int64)))
    return ok and bool(np.array_equal(orig[idx], keys))


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); ms itself without a
    process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n: int, world: int, ms_max: float) -> float:
    """Whole-job GKeys/s: every rank sorts its own n keys; the job takes the
    slowest rank's time."""
    return world * n / (ms_max * 1e-3) / 1e9


def run_reference(args):
    """Reference arm: the CPU oracle, each step a bounded sample of the workload."""
    kdt = np.uint64 if args.key == "u64" else np.uint32
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_0811_3448_gb300 import inputs
    cores = os.cpu_count() or 1
    log2g = max(0, int(math.floor(math.log2(cores))))
    # calibrate the sample so that warmup + steps take about 90 s
    probe = 1 << 20
    k = inputs.config2_keys(probe, kdt, args.dist)
    v = inputs.index_payload(probe)
    t0 = time.perf_counter()
    oracle.binar_sort_parallel(k, v, log2_groups=log2g)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    per_step = 90.0 / max(1, args.steps + args.warmup)
    n = int(min(args.n, max(1 << 18, rate * per_step)))
    keys = inputs.config2_keys(n, kdt, args.dist)
    vals = inputs.index_payload(n)
    times = []
    valid = True
    for i in range(args.warmup + args.steps):
        kk, vv = keys.copy(), vals.copy()
        t0 = time.perf_counter()
        oracle.binar_sort_parallel(kk, vv, log2_groups=log2g)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
        if i == 0 or i == args.warmup + args.steps - 1:
            valid &= host_sorted_pairs(keys, kk, vv)
    ms = 1e3 * statistics.mean(times)
    value = n / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.key, "data": "synthetic",
           "config": {"workload": workload_name(args.n, args.key, args.dist), "n": args.n, "sample_n": n, "dist": args.dist,
                      "parallelism": "replicas"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1 << log2g, "kind": "oracle",
                            "sample": f"{n} keys per step (bounded sample of the {args.n}-key "
                                      f"workload), parallel binar sort on host cores",
                            "validated": valid},
           "validated": valid,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def check_sorted_stable(tk, tv, orig_keys_dev):
    """Sorted, a permutation of the input, and stable (payload = index)."""
    import torch
    if tk.dtype == torch.uint64:   # compare as unsigned: flip the sign bit of the int64 view
        flip = torch.tensor(-(2 ** 63), dtype=torch.int64, device=tk.device)
        k = tk.view(torch.int64) ^ flip
        orig = orig_keys_dev.view(torch.int64) ^ flip
    else:
        k = tk.to(torch.int64)
        orig = orig_keys_dev.to(torch.int64)
    v = tv.to(torch.int64)
    ok = bool((k[1:] >= k[:-1]).all())
    ok &= bool((orig[v] == k).all())
    ok &= bool((torch.bincount(v, minlength=k.shape[0]) == 1).all())
    eq = k[1:] == k[:-1]
    ok &= bool((v[1:][eq] > v[:-1][eq]).all())
    return ok


def keys_only_partition_roofline(binding, torch, keys0, keys, kb, n, peak, peak_src, steps=20):
    """partition[0] of a keys-only sort of the same keys, timed with the
    library's per-kernel events over `steps` sorts."""
    ws = binding.workspace(n, kb, 0, device=keys0.device)
    for _ in range(3):
        keys.copy_(keys0)
        binding.sort_keys(keys, ws=ws)
    torch.cuda.synchronize()
    binding.profile_start()
    for _ in range(steps):
        keys.copy_(keys0)
        binding.sort_keys(keys, ws=ws)
    st = binding.profile_stop()
    binding.check_status(ws)
    ok = bool((keys[1:].to(torch.int64) >= keys[:-1].to(torch.int64)).all()) if kb == 4 else None
    part = st.get("partition[0]")
    if not part:
        return None
    per_launch_ms = part[1] / part[0]
    alg = 2 * kb * n
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    total = sum(t for _, t in st.values()) / steps
    return {"bound": "hbm", "kernel": "partition[0] (keys only)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst)",
            "algorithmic_bytes_per_launch": alg, "frac_of_8TBs_spec": achieved / 8000.0,
            "ms_per_launch": per_launch_ms, "sort_ms": total,
            "sort_gkeys_per_s": n / (total * 1e-3) / 1e9, "validated": ok}


def small_sort(binding, torch, dev, n: int = 1 << 20, reps: int = 50):
    """The 1,048,576 uniform uint32 keys of the small configuration, sorted by
    binar_sort_keys (32 bit levels): 4 MiB, resident in L2 and bound by launch
    latency, so its roofline fraction is not meaningful.  Timed per call with
    CUDA events, as stream launches and as one CUDA-graph replay of the call."""
    from paper_0811_3448_gb300 import inputs
    keys_h = inputs.config1_keys(n)
    k0 = torch.from_numpy(keys_h).to(dev)
    k = torch.empty_like(k0)
    ws = binding.workspace(n, 4, 0, device=dev)
    stream = torch.cuda.current_stream()

    def timed(run):
        ts = []
        for i in range(reps + 3):
            k.copy_(k0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    ms = timed(lambda: binding.sort_keys(k, ws=ws))
    binding.check_status(ws)
    ok = bool(torch.equal(k.cpu(), torch.from_numpy(np.sort(keys_h))))
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            binding.sort_keys(k, ws=ws)
    stream.wait_stream(cap)
    gms = timed(graph.replay)
    binding.check_status(ws)
    ok &= bool(torch.equal(k.cpu(), torch.from_numpy(np.sort(keys_h))))
    return {"workload": f"{n} uniform uint32 keys, keys only (binar_sort_keys)", "n": n,
            "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_median": ms,
            "graph_value": n / (gms * 1e-3) / 1e9, "graph_ms_median": gms,
            "validated": ok, "l2": "4 MiB input, L2-resident (launch-bound; no roofline)"}


def run_e2e(args, binding, torch, dev, keys_h, vals_h, ws, keys, vals, world):
    """End-to-end throughput through the public API with pinned host buffers.

    Every step copies its inputs host -> device, sorts them with
    binding.sort_pairs and copies the sorted keys and payloads device -> host,
    all inside the timed region.  Streamed: three device buffer sets and three
    streams (copy in, sort, copy out), so step i's copy out overlaps step i+1's
    copy in and sort, as for a caller sorting a stream of arrays (three buffer
    sets keep both link directions busy).  The serial
    form (copy in, sort, copy out, one step at a time) is reported beside it."""
    n = keys_h.shape[0]
    rec = keys_h.itemsize + vals_h.itemsize      # bytes per record each way
    hk = torch.from_numpy(keys_h).pin_memory()
    hv = torch.from_numpy(vals_h).pin_memory()
    ok_k = torch.empty_like(hk).pin_memory()
    ok_v = torch.empty_like(hv).pin_memory()
    steps = max(2, args.e2e_steps)
    # first use of freshly pinned buffers maps them for the device (a one-time
    # cost of hundreds of ms): one untimed copy each way
    keys.copy_(hk, non_blocking=True)
    vals.copy_(hv, non_blocking=True)
    ok_k.copy_(keys, non_blocking=True)
    ok_v.copy_(vals, non_blocking=True)
    torch.cuda.synchronize()
    # streamed
    nbuf = 3
    bk = [keys] + [torch.empty_like(keys) for _ in range(nbuf - 1)]
    bv = [vals] + [torch.empty_like(vals) for _ in range(nbuf - 1)]
    s_in, s_sort, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    copied_in = [torch.cuda.Event() for _ in range(steps)]
    sorted_ = [torch.cuda.Event() for _ in range(steps)]
    copied_out = [torch.cuda.Event() for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(s_in)
    for i in range(steps):
        b = i % nbuf
        with torch.cuda.stream(s_in):
            if i >= nbuf:
                s_in.wait_event(copied_out[i - nbuf])    # buffer b is free again
            bk[b].copy_(hk, non_blocking=True)
            bv[b].copy_(hv, non_blocking=True)
            copied_in[i].record(s_in)
        with torch.cuda.stream(s_sort):
            s_sort.wait_event(copied_in[i])
            binding.sort_pairs(bk[b], bv[b], ws=ws, stream=s_sort)
            sorted_[i].record(s_sort)
        with torch.cuda.stream(s_out):
            s_out.wait_event(sorted_[i])
            ok_k.copy_(bk[b], non_blocking=True)
            ok_v.copy_(bv[b], non_blocking=True)
            copied_out[i].record(s_out)
    s_out.wait_event(copied_out[steps - 1])
    t1.record(s_out)
    t1.synchronize()
    binding.check_status(ws, stream=s_sort)
    ms = t0.elapsed_time(t1) / steps
    # serial
    stream = torch.cuda.current_stream()
    serial = []
    for i in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        keys.copy_(hk, non_blocking=True)
        vals.copy_(hv, non_blocking=True)
        binding.sort_pairs(keys, vals, ws=ws)
        ok_k.copy_(keys, non_blocking=True)
        ok_v.copy_(vals, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            serial.append(e0.elapsed_time(e1))
    binding.check_status(ws)
    ser = statistics.mean(serial)
    return {"value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": rec * n, "d2h_bytes_per_step": rec * n, "ms_per_step": ms,
            "steps": steps, "form": "streamed: step i's copy out overlaps later steps' copy in "
                                    "and sort (three device buffer sets)",
            "serial": {"value": world * n / (ser * 1e-3) / 1e9, "ms_per_step": ser}}


def run_binar(args):
    import torch
    from paper_0811_3448_gb300 import binding, inputs

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    binding.load()
    dev = torch.device("cuda", local)
    n = args.n
    kb = 8 if args.key == "u64" else 4
    kdt = np.uint64 if kb == 8 else np.uint32

    keys_h = inputs.config2_keys(n, kdt, args.dist)
    vals_h = inputs.index_payload(n)
    keys0 = torch.from_numpy(keys_h).to(dev)
    vals0 = torch.from_numpy(vals_h).to(dev)
    keys = torch.empty_like(keys0)
    vals = torch.empty_like(vals0)
    ws = binding.workspace(n, kb, 4, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        keys.copy_(keys0)
        vals.copy_(vals0)
        binding.sort_pairs(keys, vals, ws=ws)
    binding.check_status(ws)

    sampler = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        keys.copy_(keys0)
        vals.copy_(vals0)
        evs[i][0].record(stream)
        binding.sort_pairs(keys, vals, ws=ws)
        evs[i][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    binding.check_status(ws)
    # the per-kernel split comes from a second loop of the same sorts with
    # every launch bracketed by CUDA events on the sort's stream, so that the
    # timed loop above runs the plain call
    prof_steps = min(args.steps, 20)
    binding.profile_start()
    for i in range(prof_steps):
        keys.copy_(keys0)
        vals.copy_(vals0)
        binding.sort_pairs(keys, vals, ws=ws)
    torch.cuda.synchronize()
    kstats = binding.profile_stop()
    sampler.stop()
    binding.check_status(ws)
    ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
    ms_max = max_over_ranks(ms, dist, dev)
    value = replica_throughput(n, world, ms_max)
    valid = check_sorted_stable(keys, vals, keys0)

    # roofline of the first partition pass (the whole array, one read + one write)
    peak, peak_src = measured_peaks()
    kernels = {}
    total_ms = sum(t for _, t in kstats.values()) or 1.0
    for name, (launches, t) in kstats.items():
        kernels[name] = {"launches": launches, "ms_per_launch": t / max(launches, 1),
                         "share": t / total_ms}
    part = kstats.get("partition[0]")
    roofline = None
    if part:
        per_launch_ms = part[1] / part[0]
        alg_bytes = 2 * (kb + 4) * n
        achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": "partition[0]", "achieved": achieved,
                    "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst)",
                    "traffic": recorded_traffic("partition[0]", kb, 4, n),
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "frac_of_8TBs_spec": achieved / 8000.0}
    dominant = max(kernels.items(), key=lambda kv: kv[1]["share"])[0] if kernels else None
    ms_median = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)

    # the same partition pass on the keys alone (unstable ranking suffices for
    # keys: equal keys are indistinguishable), against 2 K n bytes
    roofline_keys = keys_only_partition_roofline(binding, torch, keys0, keys, kb, n, peak, peak_src,
                                                 steps=min(args.steps, 20))
    launches_per_sort = sum(l for l, _ in kstats.values()) / max(prof_steps, 1)
    gpu_launches = int(round(launches_per_sort * args.steps))
    instrumented_ms = sum(t for _, t in kstats.values()) / max(prof_steps, 1)

    # end to end through the public API: pinned host buffers, copies inside the timed region
    e2e = run_e2e(args, binding, torch, dev, keys_h, vals_h, ws, keys, vals, world)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.key, "data": "synthetic",
           "config": {"workload": workload_name(n, args.key, args.dist), "n": n,
                      "key": "uint64" if kb == 8 else "uint32", "payload": "uint32",
                      "dist": args.dist, "parallelism": f"replicas x{world}",
                      "l2": "2 GiB inputs (> 129 MB L2), restored from a pristine copy "
                            "before every timed sort"},
           "e2e": e2e, "roofline": roofline, "gpu_launches": gpu_launches,
           "clocks": sampler.summary(), "validated": valid, "dominant_kernel": dominant,
           "kernels": kernels, "wall_s_timed_loop": wall, "ms_median": ms_median,
           "kernel_split": {"steps": prof_steps, "form": "separate loop, every launch "
                            "bracketed by CUDA events on the sort's stream",
                            "sum_of_kernels_ms": instrumented_ms},
           "roofline_keys_only": roofline_keys,
           "config1": small_sort(binding, torch, dev)}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(32 << 20, args.dist, kdt)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def check_segments_sorted(torch, off, k_in, k_out, v_out):
    """Every segment sorted, payload (index within the segment) a permutation
    of the segment pointing at the key it came with, equal keys in input order."""
    n = k_out.shape[0]
    seg = torch.repeat_interleave(torch.arange(off.shape[0] - 1, device=off.device),
                                  off[1:] - off[:-1])
    k = k_out.to(torch.int64)
    v = v_out.to(torch.int64)
    same = seg[1:] == seg[:-1]
    ok = bool((k[1:][same] >= k[:-1][same]).all())
    gidx = off[:-1][seg] + v
    ok &= bool((torch.bincount(gidx, minlength=n) == 1).all())
    ok &= bool((k_in.to(torch.int64)[gidx] == k).all())
    eq = same & (k[1:] == k[:-1])
    ok &= bool((v[1:][eq] > v[:-1][eq]).all())
    return ok


def run_segments(args):
    """Config 4: 20,000 log-uniform segments (~256M uint32 keys, uint32 payload =
    index within the segment), the whole segmented sort captured as one CUDA
    graph and replayed; compared with one binar_sort_pairs call per segment."""
    import torch
    from paper_0811_3448_gb300 import autotune, binding, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if args.seg_len > 0:
        sizes = np.full(max(1, args.n // args.seg_len), args.seg_len, dtype=np.int64)
    else:
        sizes = inputs.config4_segment_sizes(total=args.n, count=20000)
    off_h = inputs.offsets_from_sizes(sizes)
    n = int(off_h[-1])
    keys_h = inputs.uniform_keys(n, np.uint32, inputs.rng(4, 1))
    b = args.seg_prefix_bits
    if 0 < b < 32:
        # every segment's keys share a top-b-bit prefix of their own
        seg_of = np.repeat(np.arange(len(sizes), dtype=np.uint64), sizes)
        prefix = (seg_of * np.uint64(0x9E3779B1)) & np.uint64((1 << b) - 1)
        keys_h = ((prefix << np.uint64(32 - b)) |
                  (keys_h.astype(np.uint64) >> np.uint64(b))).astype(np.uint32)
    vals_h = inputs.segment_index_payload(off_h)
    dev = torch.device("cuda", local)
    off = torch.from_numpy(off_h).to(dev)
    k0 = torch.from_numpy(keys_h).to(dev)
    v0 = torch.from_numpy(vals_h).to(dev)
    k, v = k0.clone(), v0.clone()
    segs = len(off_h) - 1
    if args.no_autotune:
        cfg, timings = binding.Config(), {}
    else:
        cfg, timings = autotune.tune(k0, v0, off)
    ws = binding.workspace(n, 4, 4, segs, device=dev)
    binding.sort_segmented(k, off, v, ws=ws, config=cfg)      # set-up before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            binding.sort_segmented(k, off, v, ws=ws, config=cfg)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        k.copy_(k0)
        v.copy_(v0)
        graph.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for i in range(args.steps):
        k.copy_(k0)
        v.copy_(v0)
        evs[i][0].record(stream)
        graph.replay()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    binding.check_status(ws)
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    valid = check_segments_sorted(torch, off, k0, k, v)
    # the plain form: one sort call per segment
    plain = None
    if not args.no_plain:
        k.copy_(k0)
        v.copy_(v0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for s_ in range(segs):
            a, b = int(off_h[s_]), int(off_h[s_ + 1])
            if b - a >= 2:
                binding.sort_pairs(k[a:b], v[a:b], ws=ws)
        e1.record(stream)
        e1.synchronize()
        plain_wall = time.perf_counter() - t0
        plain_ms = e0.elapsed_time(e1)
        binding.check_status(ws)
        plain = {"value": n / (plain_ms * 1e-3) / 1e9, "unit": UNIT, "ms": plain_ms,
                 "wall_s": plain_wall, "calls": segs}
    out = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic",
           "config": {"workload": (f"{segs} segments of {args.seg_len} keys" if args.seg_len > 0 else
                                   "20,000 segments, log-uniform sizes in [1, 2^20] rescaled to")
                                  + f" {n} uint32 keys + uint32 payload, one CUDA-graph launch"
                                  + (f", keys of a segment sharing their top {args.seg_prefix_bits} bits"
                                     if 0 < args.seg_prefix_bits < 32 else ""),
                      "segments": segs, "n": n, "parallelism": f"replicas x{world}",
                      "l2": "1 GiB keys + 1 GiB payloads restored before every replay"},
           "autotuned": {"tile_keys": cfg.tile_keys, "bits_per_pass": cfg.bits_per_pass,
                         "small_cutoff": cfg.small_cutoff, "candidates": len(timings),
                         "timings_ms": timings},
           "plain_per_segment": plain, "validated": valid,
           "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_inplace(args):
    """The pairs workload sorted by binar_sort_inplace (unstable, no second
    array), timed like the headline; reports the workspace beside the
    out-of-place sort's."""
    import torch
    from paper_0811_3448_gb300 import binding, inputs
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    kb = 8 if args.key == "u64" else 4
    kdt = np.uint64 if kb == 8 else np.uint32
    keys0 = torch.from_numpy(inputs.config2_keys(n, kdt, args.dist)).to(dev)
    vals0 = torch.from_numpy(inputs.index_payload(n)).to(dev)
    keys, vals = torch.empty_like(keys0), torch.empty_like(vals0)
    wsb = binding.inplace_workspace_bytes(n, kb, 4)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        keys.copy_(keys0)
        vals.copy_(vals0)
        binding.sort_inplace(keys, vals, ws=ws)
    binding.check_status(ws)
    sampler = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for i in range(args.steps):
        keys.copy_(keys0)
        vals.copy_(vals0)
        evs[i][0].record(stream)
        binding.sort_inplace(keys, vals, ws=ws)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    binding.check_status(ws)
    binding.profile_start()
    for i in range(min(args.steps, 3)):
        keys.copy_(keys0)
        vals.copy_(vals0)
        binding.sort_inplace(keys, vals, ws=ws)
    torch.cuda.synchronize()
    kst = binding.profile_stop()
    sampler.stop()
    binding.check_status(ws)
    per = {}
    for name, (launches, t) in kst.items():      # summed over the levels, per sort
        base = name.split("[")[0]
        per[base] = per.get(base, 0.0) + t / min(args.steps, 3)
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    ref = keys0.clone()
    binding.sort_keys(ref)
    vv = vals.to(torch.int64)
    valid = bool(torch.equal(keys, ref)) and bool((torch.bincount(vv, minlength=n) == 1).all()) \
        and bool(torch.equal(keys0.to(torch.int64)[vv], keys.to(torch.int64)))
    out = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.key,
           "data": "synthetic",
           "config": {"workload": workload_name(n, args.key, args.dist).replace(
                          "stable in-place sort", "unstable in-place mode (one bit per level)"),
                      "n": n, "parallelism": "replicas x1",
                      "l2": "inputs > 129 MB L2, restored from a pristine copy before every sort"},
           "workspace_bytes": wsb, "out_of_place_workspace_bytes": binding.workspace_bytes(n, kb, 4),
           "kernels_ms_per_sort": {k: round(v, 4) for k, v in sorted(per.items(), key=lambda x: -x[1])},
           "validated": valid, "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "segments":
        run_segments(args)
    elif args.workload == "inplace":
        run_inplace(args)
    elif args.workload == "serve":
        from paper_0811_3448_gb300 import serve
        sampler = ClockSampler(dist_env()[2])
        sampler.start()
        line = serve.bench_main(args)
        sampler.stop()
        if line is not None:
            line["clocks"] = sampler.summary()
            print(json.dumps(line), flush=True)
    else:
        run_binar(args)


if __name__ == "__main__":
    main()
