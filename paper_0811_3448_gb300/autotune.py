"""Autotuner for libbinar's tunable parameters.

The knobs are those of ``binar_config``: the partition tile (keys per tile:
two compiled shapes per key and payload width), the key bits fused per
partition pass k (6, 7 or 8: fewer bits make more, smaller levels and a
different bucket-size spread at the finisher) and the small-bucket cutoff C
(buckets of at most C keys finish in shared memory).  Persistent CTAs per SM
stay at each kernel's occupancy.  The tuner times every candidate on
the caller's own data with CUDA events (a few repetitions after a warm-up,
inputs restored between runs) and keeps the fastest.  Results are cached in a
JSON file (``$BINAR_TUNE_CACHE`` or ``~/.cache/libbinar/tune.json``) keyed by
GPU name, key and payload width, log2 of the key count and the number of
segments, so the cost is paid once per shape class.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("BINAR_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "libbinar", "tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass   # a read-only home is not an error: the result is just not kept


def shape_key(n: int, key_bytes: int, val_bytes: int, num_segments: int = 0,
              device_name: str = None) -> str:
    dev = torch.cuda.get_device_name() if device_name is None else device_name
    seg_class = 0 if num_segments <= 1 else int(math.log2(num_segments)) + 1
    return f"{dev}|k{key_bytes}|v{val_bytes}|n2^{max(0, int(math.log2(max(n, 1))))}|s{seg_class}"


BITS = (6, 7, 8)


def candidates(key_bytes: int, val_bytes: int = 0):
    """Every (tile, bits per pass, small cutoff) the library accepts for the shape."""
    cap = {4: 8192, 8: 4096, 16: 2048}[key_bytes]
    cutoffs = [c for c in (2048, 4096, 8192) if c <= cap]
    return [binding.Config(tile_keys=t, bits_per_pass=b, small_cutoff=c)
            for t in binding.tile_choices(key_bytes, val_bytes) for b in BITS for c in cutoffs]


def describe(cfg) -> str:
    return f"tile={cfg.tile_keys},bits={cfg.bits_per_pass},cutoff={cfg.small_cutoff}"


def _as_dict(cfg) -> dict:
    return {"tile_keys": cfg.tile_keys, "bits_per_pass": cfg.bits_per_pass,
            "small_cutoff": cfg.small_cutoff}


def _time(run, restore, reps: int = 3) -> float:
    stream = torch.cuda.current_stream()
    best = float("inf")
    restore()
    run()   # warm-up (and first-call set-up)
    for _ in range(reps):
        restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(keys: torch.Tensor, vals: torch.Tensor = None, offsets: torch.Tensor = None,
         key_map=None, use_cache: bool = True, reps: int = 3):
    """Returns (best binar_config, {description: ms}) for sorting these inputs
    (segmented if ``offsets`` is given).  The inputs are not modified."""
    n, kb, _ = binding.key_layout(keys)
    vb = 0 if vals is None else vals.element_size()
    segs = 0 if offsets is None else offsets.shape[0] - 1
    key = shape_key(n, kb, vb, segs)
    with _lock:
        cache = _load_cache() if use_cache else {}
        hit = cache.get(key)
    if hit is not None and set(hit.get("config", {})) == set(_as_dict(binding.Config())):
        return binding.Config(**hit["config"]), hit.get("timings", {})
    work_k = torch.empty_like(keys)
    work_v = None if vals is None else torch.empty_like(vals)
    ws = binding.workspace(n, kb, vb, max(segs, 1), device=keys.device)

    def restore():
        work_k.copy_(keys)
        if vals is not None:
            work_v.copy_(vals)

    timings, best, best_ms = {}, None, float("inf")
    for cfg in candidates(kb, vb):
        if offsets is not None:
            run = lambda: binding.sort_segmented(work_k, offsets, work_v, key_map=key_map, ws=ws,
                                                 config=cfg)
        elif vals is not None:
            run = lambda: binding.sort_pairs(work_k, work_v, key_map=key_map, ws=ws, config=cfg)
        else:
            run = lambda: binding.sort_keys(work_k, key_map=key_map, ws=ws, config=cfg)
        ms = _time(run, restore, reps)
        binding.check_status(ws)
        timings[describe(cfg)] = ms
        if ms < best_ms:
            best, best_ms = cfg, ms
    entry = {"config": _as_dict(best), "ms": best_ms, "timings": timings}
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = entry
            _store_cache(cache)
    return best, timings
