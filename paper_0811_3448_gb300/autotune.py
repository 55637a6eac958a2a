"""Autotuner for libbinar's tunable parameters.

The knobs are those of ``binar_config``: the small-bucket cutoff C, the number
of persistent partition CTAs per SM and the partition tile (keys per tile;
one compiled choice per key width today).  The tuner times every candidate on
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


def candidates(key_bytes: int):
    """Every (small_cutoff, ctas_per_sm) pair the library accepts for the key width."""
    cap = {4: 8192, 8: 4096, 16: 2048}[key_bytes]
    cutoffs = [c for c in (2048, 4096, 8192) if c <= cap]
    return [binding.Config(small_cutoff=c, ctas_per_sm=k) for c in cutoffs for k in (0, 1, 2)]


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
    if hit is not None:
        return binding.Config(**hit["config"]), hit.get("timings", {})
    work_k = torch.empty_like(keys)
    work_v = None if vals is None else torch.empty_like(vals)
    ws = binding.workspace(n, kb, vb, max(segs, 1), device=keys.device)

    def restore():
        work_k.copy_(keys)
        if vals is not None:
            work_v.copy_(vals)

    timings, best, best_ms = {}, None, float("inf")
    for cfg in candidates(kb):
        if offsets is not None:
            run = lambda: binding.sort_segmented(work_k, offsets, work_v, key_map=key_map, ws=ws,
                                                 config=cfg)
        elif vals is not None:
            run = lambda: binding.sort_pairs(work_k, work_v, key_map=key_map, ws=ws, config=cfg)
        else:
            run = lambda: binding.sort_keys(work_k, key_map=key_map, ws=ws, config=cfg)
        ms = _time(run, restore, reps)
        binding.check_status(ws)
        desc = f"cutoff={cfg.small_cutoff},ctas_per_sm={cfg.ctas_per_sm}"
        timings[desc] = ms
        if ms < best_ms:
            best, best_ms = cfg, ms
    entry = {"config": {"small_cutoff": best.small_cutoff, "ctas_per_sm": best.ctas_per_sm},
             "ms": best_ms, "timings": timings}
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = entry
            _store_cache(cache)
    return best, timings
