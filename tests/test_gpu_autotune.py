"""Autotuner on the GPU: picks one of the candidates, caches it, and the
chosen configuration sorts correctly."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import autotune, binding, inputs

pytestmark = pytest.mark.gpu


def test_tune_pairs_and_cache(tmp_path, monkeypatch):
    require_gpu()
    monkeypatch.setenv("BINAR_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 1 << 20
    keys = inputs.uniform_keys(n, np.uint32, inputs.rng(2, 7))
    vals = inputs.index_payload(n)
    tk, tv = to_dev(keys), to_dev(vals)
    cfg, timings = autotune.tune(tk, tv, reps=2)
    assert (cfg.small_cutoff, cfg.ctas_per_sm) in {(c.small_cutoff, c.ctas_per_sm)
                                                   for c in autotune.candidates(4)}
    assert len(timings) == len(autotune.candidates(4)) and all(t > 0 for t in timings.values())
    # inputs untouched
    assert same_bits(to_host(tk), keys) and same_bits(to_host(tv), vals)
    cfg2, timings2 = autotune.tune(tk, tv)                  # served from the cache
    assert (cfg2.small_cutoff, cfg2.ctas_per_sm) == (cfg.small_cutoff, cfg.ctas_per_sm)
    assert timings2 == timings
    binding.sort_pairs(tk, tv, config=cfg)
    ek, ev = keys.copy(), vals.copy()
    oracle.stable_radix(ek, ev)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)
