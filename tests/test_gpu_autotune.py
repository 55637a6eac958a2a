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
    cands = autotune.candidates(4, 4)
    assert autotune.describe(cfg) in {autotune.describe(c) for c in cands}
    assert set(timings) == {autotune.describe(c) for c in cands}
    assert all(t > 0 for t in timings.values())
    # inputs untouched
    assert same_bits(to_host(tk), keys) and same_bits(to_host(tv), vals)
    cfg2, timings2 = autotune.tune(tk, tv)                  # served from the cache
    assert autotune.describe(cfg2) == autotune.describe(cfg)
    assert timings2 == timings
    binding.sort_pairs(tk, tv, config=cfg)
    ek, ev = keys.copy(), vals.copy()
    oracle.stable_radix(ek, ev)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)


@pytest.mark.parametrize("tile_variant", [0, 1])
@pytest.mark.parametrize("bits", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind", ["uint32", "uint64", "b16"])
def test_every_tile_and_width_sorts_like_the_oracle(tile_variant, bits, kind):
    """Each point of the tuner's space (and the smaller k it does not search)
    gives the oracle's stable order: keys alone, pairs and segments."""
    require_gpu()
    n = 300_001
    g = np.random.Generator(np.random.PCG64(bits + 10 * tile_variant))
    if kind == "b16":
        keys = g.integers(0, 256, size=(n, 16), dtype=np.uint8)
        keys[::3] = keys[0]
        kmap, kb = binding.MAP_BYTES_BE, 16
    else:
        keys = inputs.uniform_keys(n, np.dtype(kind), g)
        keys[::3] = keys[0]
        kmap, kb = binding.MAP_UNSIGNED, keys.itemsize
    vals = inputs.index_payload(n)
    for vb in (0, 4):
        cfg = {"tile_keys": binding.tile_choices(kb, vb)[tile_variant], "bits_per_pass": bits,
               "small_cutoff": 2048}
        tk = to_dev(keys)
        ws = binding.workspace(n, kb, vb)
        if vb == 0:
            binding.sort_keys(tk, key_map=kmap, config=cfg, ws=ws)
            binding.check_status(ws)
            ek = keys.copy()
            oracle.binar_sort(ek, key_map=kmap)
            assert same_bits(to_host(tk), ek)
        else:
            tv = to_dev(vals)
            binding.sort_pairs(tk, tv, key_map=kmap, config=cfg, ws=ws)
            binding.check_status(ws)
            ek, ev = keys.copy(), vals.copy()
            oracle.stable_radix(ek, ev, key_map=kmap)
            assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)
    off = inputs.offsets_from_sizes(np.array([5, 70000, 0, 200000, 29996], dtype=np.int64))
    assert off[-1] == n
    tk, tv = to_dev(keys), to_dev(vals)
    cfg = {"tile_keys": binding.tile_choices(kb, 4)[tile_variant], "bits_per_pass": bits}
    ws = binding.workspace(n, kb, 4, len(off) - 1)
    binding.sort_segmented(tk, to_dev(off), tv, key_map=kmap, config=cfg, ws=ws)
    binding.check_status(ws)
    ek, ev = keys.copy(), vals.copy()
    oracle.stable_radix(ek, ev, key_map=kmap, offsets=off)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)


@pytest.mark.parametrize("bits", [1, 3, 5, 8])
@pytest.mark.parametrize("pos", [0, 7, 29])
def test_partition_pass_of_any_width(bits, pos):
    """One stable pass on 1 .. 8 bits; bits = 1 is the paper's partition step
    ("Partition Array into Sub-arrays": lower sub-array for bit 0, upper for
    bit 1), here stable."""
    require_gpu()
    n = 100_003
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(pos + bits)))
    vals = inputs.index_payload(n)
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=pos, bits=bits)
    ek, ev, eoffs = oracle.partition_pass(keys, vals, pos=pos, k=bits)
    assert same_bits(to_host(ko), ek) and same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)
