"""Serving loop: sort requests of mixed sizes and key types, admitted under a
device-memory budget and continuously batched into segmented launches.

Structure (one host thread, CUDA streams for overlap):

* :class:`Arena` -- the device-memory budget.  One device buffer of
  ``budget_bytes`` is carved first-fit into 256-byte aligned blocks; a batch
  holds one block (its keys, payloads, offsets and workspace) from launch
  until its completion event has fired.  Admission is exactly "the block fits".
* :class:`Scheduler` -- host logic only.  Requests wait in arrival order (one
  deque per class).  When a stream slot is free, the oldest request picks the
  class (key type, payload or not); queued requests of that class join the
  batch, in arrival order,
  while the batch stays under ``max_batch_keys`` / ``max_batch_requests`` and
  its block fits the arena's largest free range.  If the oldest request does
  not fit, nothing launches until memory frees (no overtaking, so no request
  starves).  A request whose block alone exceeds the whole budget is rejected
  at arrival.
* :class:`Server` -- the device side.  A batch's inputs are written into its
  block (``binar_generate``, standing in for the client's producer), the whole
  batch is one ``binar_sort_segmented`` call on the slot's stream (a batch of
  one request is sorted by ``binar_sort_pairs`` / ``binar_sort_keys`` directly,
  without the offsets copy and the segment seeding), and an event marks
  completion.  With ``linger_s`` > 0 a batch smaller than ``linger_keys`` waits
  up to ``linger_s`` after its oldest request arrived, while other batches are
  in flight, for more requests of its class to join.  Requests that arrive while batches run are admitted as
  slots and memory free up, so batches of different classes overlap on the
  device.  ``mode="plain"`` is the comparison form: one request per launch
  (``binar_sort_pairs`` / ``binar_sort_keys``), same slots and budget.

Latency of a request = time its completion was observed on the host - its
arrival time (both on the host's monotonic clock).
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import math
import os
import time
from typing import Callable, List, Optional

import numpy as np

ALIGN = 256
KEY_BYTES = {"u32": 4, "u64": 8, "f32": 4}


def _align(x: int, a: int = ALIGN) -> int:
    return -(-x // a) * a


class Arena:
    """First-fit allocator of [0, capacity) in ``align``-byte units."""

    def __init__(self, capacity: int, align: int = ALIGN):
        self.align = align
        self.capacity = capacity - capacity % align
        self.free_list = [(0, self.capacity)] if self.capacity > 0 else []
        self.live = {}
        self.used = 0
        self.peak = 0

    def alloc(self, nbytes: int) -> Optional[int]:
        size = max(self.align, _align(nbytes, self.align))
        for i, (off, sz) in enumerate(self.free_list):
            if sz >= size:
                if sz == size:
                    del self.free_list[i]
                else:
                    self.free_list[i] = (off + size, sz - size)
                self.live[off] = size
                self.used += size
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off: int) -> None:
        size = self.live.pop(off)
        self.used -= size
        i = bisect.bisect_left(self.free_list, (off, 0))
        if i < len(self.free_list) and off + size == self.free_list[i][0]:
            size += self.free_list[i][1]
            del self.free_list[i]
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == off:
            self.free_list[i - 1] = (self.free_list[i - 1][0], self.free_list[i - 1][1] + size)
        else:
            self.free_list.insert(i, (off, size))

    def largest_free(self) -> int:
        return max((s for _, s in self.free_list), default=0)


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    key_type: str            # "u32" | "u64" | "f32"
    has_payload: bool        # uint32 payload = index within the request
    seed: int                # SplitMix64 seed of the request's keys
    arrival_s: float = 0.0
    _seq: int = -1           # submission number (set by the scheduler)
    status: str = "new"      # queued, running, done, rejected, failed
    t_launch: float = math.nan
    t_done: float = math.nan
    error: str = ""

    @property
    def cls(self):
        return (self.key_type, self.has_payload)

    @property
    def key_bytes(self) -> int:
        return KEY_BYTES[self.key_type]

    @property
    def val_bytes(self) -> int:
        return 4 if self.has_payload else 0

    @property
    def latency_s(self) -> float:
        return self.t_done - self.arrival_s


@dataclasses.dataclass
class BlockLayout:
    n: int
    keys_off: int
    vals_off: int
    offs_off: int
    ws_off: int
    ws_bytes: int
    total: int


def block_layout(sizes: List[int], key_bytes: int, val_bytes: int,
                 ws_bytes: Callable[[int, int, int, int], int]) -> BlockLayout:
    """Byte layout of one batch's block: keys | payloads | offsets | workspace."""
    n = int(sum(sizes))
    keys_off = 0
    vals_off = _align(n * key_bytes)
    offs_off = _align(vals_off + n * val_bytes)
    ws_off = _align(offs_off + 8 * (len(sizes) + 1))
    wb = int(ws_bytes(n, key_bytes, val_bytes, max(len(sizes), 1)))
    return BlockLayout(n, keys_off, vals_off, offs_off, ws_off, wb, _align(ws_off + wb))


@dataclasses.dataclass
class Batch:
    cls: tuple
    requests: List[Request]
    layout: BlockLayout
    arena_off: int
    starts: List[int]
    slot: int = -1
    event: object = None


class Scheduler:
    """Admission and batch formation (host logic only, no device calls).

    Queued requests wait in one deque per class, in arrival order; the oldest
    request overall (smallest submission number) picks the class of the next
    batch.  Forming a batch costs O(classes + batch size), however long the
    backlog."""

    def __init__(self, arena: Arena, ws_bytes, max_batch_keys: int = 256 << 20,
                 max_batch_requests: int = 4096):
        self.arena = arena
        self.ws_bytes = ws_bytes
        self.max_batch_keys = max_batch_keys
        self.max_batch_requests = max_batch_requests
        self.queues = {}
        self.rejected: List[Request] = []
        self._seq = 0
        self._queued = 0

    @property
    def queued(self) -> int:
        return self._queued

    @property
    def queue(self) -> List[Request]:
        """All queued requests in submission order (for inspection)."""
        return sorted((r for q in self.queues.values() for r in q), key=lambda r: r._seq)

    def submit(self, r: Request) -> bool:
        if block_layout([r.n], r.key_bytes, r.val_bytes, self.ws_bytes).total > self.arena.capacity:
            r.status = "rejected"
            r.error = "larger than the device-memory budget"
            self.rejected.append(r)
            return False
        r.status = "queued"
        r._seq = self._seq
        self._seq += 1
        self.queues.setdefault(r.cls, collections.deque()).append(r)
        self._queued += 1
        return True

    def next_batch(self) -> Optional[Batch]:
        if self._queued == 0:
            return None
        q = min((q for q in self.queues.values() if q), key=lambda q: q[0]._seq)
        head = q[0]
        kb, vb = head.key_bytes, head.val_bytes
        room = self.arena.largest_free()
        sizes, layout, total = [], None, 0
        for r in q:
            if len(sizes) >= self.max_batch_requests:
                break
            if sizes and total + r.n > self.max_batch_keys:
                break
            trial = block_layout(sizes + [r.n], kb, vb, self.ws_bytes)
            if trial.total > room:
                break
            sizes.append(r.n)
            total += r.n
            layout = trial
        if not sizes:
            return None          # the oldest request waits for memory
        off = self.arena.alloc(layout.total)
        assert off is not None
        chosen = [q.popleft() for _ in range(len(sizes))]
        self._queued -= len(chosen)
        starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64).tolist()
        return Batch(head.cls, chosen, layout, off, starts)

    def should_linger(self, now: float, linger_s: float, linger_keys: int) -> bool:
        """True while the next batch would be small (its class holds fewer
        than ``linger_keys`` queued keys) and its oldest request arrived less
        than ``linger_s`` ago: waiting lets more requests of the class join."""
        if self._queued == 0:
            return False
        q = min((q for q in self.queues.values() if q), key=lambda q: q[0]._seq)
        if now - q[0].arrival_s >= linger_s:
            return False
        total = 0
        for r in q:
            total += r.n
            if total >= linger_keys:
                return False
        return True

    def release(self, batch: Batch) -> None:
        self.arena.free(batch.arena_off)


def percentile(xs, q):
    if not xs:
        return None
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


class Server:
    """Runs a list of requests in real time against the GPU.

    mode: "batched" (continuous batching into segmented launches) or "plain"
    (one request per launch).  ``keep(r)`` selects requests whose sorted
    output is copied out (for checking) before their block is released."""

    def __init__(self, budget_bytes: int = 40 << 30, slots: int = 4, mode: str = "batched",
                 max_batch_keys: int = 256 << 20, max_batch_requests: int = 4096,
                 device=None, config=None, linger_s: float = 0.0, linger_keys: int = 1 << 20):
        import torch
        from . import binding
        if mode not in ("batched", "plain"):
            raise ValueError(f"unknown mode {mode}")
        self.torch, self.binding = torch, binding
        self.mode = mode
        self.linger_s = linger_s if mode == "batched" else 0.0
        self.linger_keys = linger_keys
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.config = config
        self.buf = torch.empty(budget_bytes - budget_bytes % ALIGN, dtype=torch.uint8,
                               device=self.device)
        self.arena = Arena(self.buf.numel())
        self.sched = Scheduler(self.arena, binding.workspace_bytes,
                               max_batch_keys if mode == "batched" else 1 << 62,
                               max_batch_requests if mode == "batched" else 1)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.free_slots = list(range(slots))
        cap = (max_batch_requests if mode == "batched" else 1) + 1
        self.staging = [torch.empty(cap, dtype=torch.int64).pin_memory() for _ in range(slots)]
        self.inflight: List[Batch] = []
        self.kept = {}
        self.batches = 0
        self.batch_sizes = []
        self.failed_launches = 0

    # -- device views of a block
    def _views(self, b: Batch):
        torch = self.torch
        L, base = b.layout, b.arena_off
        kt, has_payload = b.cls
        kdtype = {"u32": torch.uint32, "u64": torch.uint64, "f32": torch.float32}[kt]
        kb = KEY_BYTES[kt]
        keys = self.buf[base + L.keys_off: base + L.keys_off + L.n * kb].view(kdtype)
        vals = self.buf[base + L.vals_off: base + L.vals_off + L.n * 4].view(torch.int32) \
            if has_payload else None
        offs = self.buf[base + L.offs_off: base + L.offs_off + 8 * (len(b.requests) + 1)] \
            .view(torch.int64)
        ws = self.buf[base + L.ws_off: base + L.ws_off + L.ws_bytes]
        return keys, vals, offs, ws

    def _launch(self, b: Batch, now: float) -> None:
        b.slot = self.free_slots.pop()
        try:
            self._enqueue(b)
        except Exception as e:    # the batch fails; its slot and memory come back
            # work the batch already enqueued on its stream (inputs generated
            # into its block, the offsets copy from the slot's pinned staging
            # buffer) must finish before the block and the slot are reused
            try:
                self.streams[b.slot].synchronize()
            except Exception:
                pass
            for r in b.requests:
                r.status = "failed"
                r.error = f"launch: {e}"
                r.t_launch = r.t_done = now
            self.sched.release(b)
            self.free_slots.append(b.slot)
            self.failed_launches += 1
            return
        for r in b.requests:
            r.status = "running"
            r.t_launch = now
        self.inflight.append(b)
        self.batches += 1
        self.batch_sizes.append(len(b.requests))

    def _enqueue(self, b: Batch) -> None:
        torch, binding = self.torch, self.binding
        s = self.streams[b.slot]
        keys, vals, offs, ws = self._views(b)
        with torch.cuda.stream(s):
            for r, a in zip(b.requests, b.starts):
                binding.generate(keys[a:a + r.n], r.seed, stream=s)
                if vals is not None:
                    torch.arange(r.n, dtype=torch.int32, device=self.device, out=vals[a:a + r.n])
            if self.mode == "batched" and len(b.requests) > 1:
                st = self.staging[b.slot]
                st[:len(b.starts)] = torch.tensor(b.starts, dtype=torch.int64)
                offs.copy_(st[:len(b.starts)], non_blocking=True)
                binding.sort_segmented(keys, offs, vals, ws=ws, config=self.config, stream=s)
            elif vals is not None:
                binding.sort_pairs(keys, vals, ws=ws, config=self.config, stream=s)
            else:
                binding.sort_keys(keys, ws=ws, config=self.config, stream=s)
            b.event = torch.cuda.Event()
            b.event.record(s)

    def _complete(self, b: Batch, now: float, keep) -> None:
        binding = self.binding
        s = self.streams[b.slot]
        keys, vals, offs, ws = self._views(b)
        status = binding.workspace_status(ws, stream=s)
        for r, a in zip(b.requests, b.starts):
            r.t_done = now
            if status != binding.OK:
                r.status = "failed"
                r.error = binding.status_string(status)
                continue
            r.status = "done"
            if keep is not None and keep(r):
                with self.torch.cuda.stream(s):
                    k = keys[a:a + r.n].clone()
                    v = None if vals is None else vals[a:a + r.n].clone()
                s.synchronize()
                self.kept[r.rid] = (k, v)
        self.sched.release(b)
        self.free_slots.append(b.slot)

    def run(self, requests: List[Request], keep=None, max_wall_s: float = 1e9) -> dict:
        """Serves ``requests`` (sorted by arrival_s) in real time; returns stats."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        t0 = time.perf_counter()
        i = 0
        while i < len(reqs) or self.sched.queued or self.inflight:
            now = time.perf_counter() - t0
            if now > max_wall_s:
                raise RuntimeError("serving run exceeded its wall-clock limit")
            while i < len(reqs) and reqs[i].arrival_s <= now:
                self.sched.submit(reqs[i])
                i += 1
            progressed = False
            for b in list(self.inflight):
                if b.event.query():
                    self.inflight.remove(b)
                    self._complete(b, time.perf_counter() - t0, keep)
                    progressed = True
            while self.free_slots:
                if self.linger_s > 0 and self.inflight and \
                        self.sched.should_linger(now, self.linger_s, self.linger_keys):
                    break
                b = self.sched.next_batch()
                if b is None:
                    break
                self._launch(b, time.perf_counter() - t0)
                progressed = True
            if not progressed:
                wait = 50e-6
                if not self.inflight and not self.sched.queued and i < len(reqs):
                    wait = max(0.0, min(reqs[i].arrival_s - now, 0.01))
                time.sleep(wait)
        return self.stats(reqs)

    def stats(self, reqs: List[Request]) -> dict:
        done = [r for r in reqs if r.status == "done"]
        lat = [r.latency_s * 1e3 for r in done]
        wait = [(r.t_launch - r.arrival_s) * 1e3 for r in done]
        keys = sum(r.n for r in done)
        span = (max(r.t_done for r in done) - min(r.arrival_s for r in reqs)) if done else 0.0
        return {"mode": self.mode, "requests": len(reqs), "done": len(done),
                "rejected": sum(r.status == "rejected" for r in reqs),
                "failed": sum(r.status == "failed" for r in reqs),
                "keys": keys, "span_s": span,
                "gkeys_per_s": keys / span / 1e9 if span > 0 else None,
                "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                "mean_ms": float(np.mean(lat)) if lat else None,
                "max_ms": max(lat) if lat else None,
                "queue_wait_p50_ms": percentile(wait, 50), "queue_wait_p99_ms": percentile(wait, 99),
                "launches": self.batches, "failed_launches": self.failed_launches,
                "mean_requests_per_launch": float(np.mean(self.batch_sizes)) if self.batch_sizes
                else None,
                "peak_budget_bytes": self.arena.peak, "budget_bytes": self.arena.capacity}


def requests_from_mix(mix) -> List[Request]:
    """Request objects from ``inputs.config5_requests`` dicts."""
    return [Request(rid=i, n=d["n"], key_type=d["key_type"], has_payload=d["has_payload"],
                    seed=d["seed"], arrival_s=d["arrival_s"]) for i, d in enumerate(mix)]


def sort_alone(r: Request, device=None, config=None):
    """The request sorted by itself (own buffers, one launch): (keys, payload)."""
    import torch
    from . import binding
    dev = device if device is not None else "cuda"
    kdtype = {"u32": torch.uint32, "u64": torch.uint64, "f32": torch.float32}[r.key_type]
    keys = torch.empty(r.n, dtype=kdtype, device=dev)
    binding.generate(keys, r.seed)
    if r.has_payload:
        vals = torch.arange(r.n, dtype=torch.int32, device=dev)
        binding.sort_pairs(keys, vals, config=config)
        return keys, vals
    binding.sort_keys(keys, config=config)
    return keys, None


def warm_up(device=None) -> None:
    """First calls of every entry point on this device (library set-up)."""
    srv = Server(budget_bytes=256 << 20, slots=2, mode="batched", device=device)
    reqs = [Request(rid=i, n=4096 + 999 * i, key_type=kt, has_payload=p, seed=i)
            for i, (kt, p) in enumerate((kt, p) for kt in KEY_BYTES for p in (False, True))]
    srv.run(reqs)
    srv = Server(budget_bytes=256 << 20, slots=2, mode="plain", device=device)
    srv.run([dataclasses.replace(r, status="new") for r in reqs])
    del srv


def bench_main(args) -> Optional[dict]:
    """bench.py --workload serve: the request mix of Poisson arrivals at
    ``args.rate`` per second for ``args.duration`` seconds, served batched and
    then one request per launch.  Returns the JSON record (None off rank 0)."""
    import torch
    from . import inputs
    if int(os.environ.get("RANK", "0")) != 0:
        return None  # one GPU per replica: the serving loop is reported by rank 0 only
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rate = getattr(args, "rate", 2000.0)
    duration = getattr(args, "duration", 60.0)
    budget = int(getattr(args, "budget_gb", 40) * (1 << 30))
    slots = getattr(args, "slots", 4)
    span = getattr(args, "span_log2", 16)
    mix = inputs.config5_requests(rate_hz=rate, duration_s=duration, span_log2=span)
    warm_up()
    torch.cuda.synchronize()
    out = {}
    plain_slots = getattr(args, "plain_slots", 0) or slots
    for mode in ("batched", "plain"):
        reqs = requests_from_mix(mix)
        srv = Server(budget_bytes=budget, slots=slots if mode == "batched" else plain_slots,
                     mode=mode, linger_s=getattr(args, "linger_us", 0.0) * 1e-6)
        sample = {r.rid for r in reqs[::max(1, len(reqs) // 16)] if r.n <= (4 << 20)}
        out[mode] = srv.run(reqs, keep=lambda r: r.rid in sample)
        # sampled check: each kept result equals the same request sorted alone
        mism = 0
        for rid in sorted(sample):
            if rid not in srv.kept:
                continue
            k, v = srv.kept[rid]
            ak, av = sort_alone(reqs[rid])
            if not torch.equal(k.view(torch.uint8), ak.view(torch.uint8)) or \
                    (v is not None and not torch.equal(v, av)):
                mism += 1
        out[mode]["slots"] = len(srv.streams)
        out[mode]["sampled_checks"] = len(srv.kept)
        out[mode]["sampled_mismatches"] = mism
        del srv
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    b, p = out["batched"], out["plain"]
    line = {"metric": "serving p50/p99 ms and GKeys/s (continuous batching)",
            "value": b["gkeys_per_s"], "unit": "GKeys/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64/f32", "data": "synthetic",
            "config": {"workload": f"serving: Poisson arrivals {rate:g}/s for {duration:g} s, "
                                   f"sizes floor(2^(10+{span}U)), key type uniform over "
                                   "{uint32, uint64, float32}, uint32 payload with p=1/2, "
                                   f"{budget >> 30} GiB budget, {slots} stream slots, "
                                   f"linger {getattr(args, 'linger_us', 0.0):g} us",
                       "requests": len(mix)},
            "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"],
            "batched": b, "plain_one_request_per_launch": p}
    return line
