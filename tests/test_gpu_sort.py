"""GPU parity: libbinar (through the C ABI) against the CPU oracle.

Keys must equal the oracle's binar sort bit for bit; pairs must equal the
oracle's stable radix sort bit for bit (keys and payloads).  Sizes span
several tiles and ragged tails; the edge cases of the method (empty and
one-key inputs, all-equal keys, pass-through levels, keys differing only in
the last bit) are covered.
"""
import numpy as np
import pytest

import oracle
from gpu_util import expect_keys, expect_pairs, key_map_of, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def gpu_sort_keys(keys, config=None):
    t = to_dev(keys)
    ws = binding.workspace(t.shape[0], binding.key_layout(t)[1], 0)
    binding.sort_keys(t, key_map=key_map_of(keys), ws=ws, config=config)
    binding.check_status(ws)
    return to_host(t)


def gpu_sort_pairs(keys, vals, config=None):
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(tk.shape[0], binding.key_layout(tk)[1], tv.element_size())
    binding.sort_pairs(tk, tv, key_map=key_map_of(keys), ws=ws, config=config)
    binding.check_status(ws)
    return to_host(tk), to_host(tv)


def make_keys(kind, n, seed=0):
    g = np.random.Generator(np.random.PCG64(1000 + seed))
    if kind == "bytes16":
        return g.integers(0, 256, size=(n, 16), dtype=np.uint8)
    if kind == "f32":
        return inputs.config3_f32(n)
    if kind == "f64":
        x = g.standard_normal(n)
        x[::17] = -0.0
        x[::29] = np.inf
        return x
    return inputs.uniform_keys(n, np.dtype(kind), g)


def test_config1_uniform_u32_keys():
    """Config 1: 1,048,576 uniform uint32 keys, against the paper's binar sort."""
    keys = inputs.config1_keys()
    assert same_bits(gpu_sort_keys(keys), expect_keys(keys))


@pytest.mark.parametrize("kind", ["uint32", "uint64", "int32", "int64", "f32", "f64", "bytes16"])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 2047, 2048, 2049, 8193, 70001, 400003])
def test_keys_against_binar_oracle(kind, n):
    keys = make_keys(kind, n, seed=n)
    assert same_bits(gpu_sort_keys(keys), expect_keys(keys))


@pytest.mark.parametrize("kind,vdtype", [("uint32", np.uint32), ("uint64", np.uint32),
                                         ("int64", np.uint64), ("f32", np.uint32),
                                         ("bytes16", np.uint64), ("uint32", np.uint64)])
@pytest.mark.parametrize("n", [1, 3, 4097, 8193, 123457, 600001])
def test_pairs_against_stable_oracle(kind, vdtype, n):
    keys = make_keys(kind, n, seed=7 * n + 1)
    if kind != "bytes16" and n > 100:
        keys[::5] = keys[0]          # many equal keys: stability is visible
    vals = np.arange(n, dtype=vdtype)
    k, v = gpu_sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek)
    assert same_bits(v, ev)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "distinct8", "sorted", "reverse"])
def test_config2_distributions_pairs(dtype, dist):
    """Config 2 recipe at 1.5M keys: payload = original index, stable order."""
    n = 1_500_000
    keys = inputs.config2_keys(n, dtype, dist)
    vals = inputs.index_payload(n)
    k, v = gpu_sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek)
    assert same_bits(v, ev)


@pytest.mark.parametrize("which", ["f32", "i64", "bytes16", "bytes16_prefix"])
def test_config3_generalized_keys(which):
    n = 600_000
    if which == "f32":
        keys = inputs.config3_f32(n)
    elif which == "i64":
        keys = inputs.config3_i64(n)
    else:
        keys = inputs.config3_bytes16(n, shared_prefix=which.endswith("prefix"))
    assert same_bits(gpu_sort_keys(keys), expect_keys(keys))
    vals = inputs.index_payload(n)
    k, v = gpu_sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)


def test_deep_levels_with_small_cutoff():
    """Small cutoff: buckets of level 0 exceed it, so level 1 partitions too."""
    n = 3_000_000
    keys = make_keys("uint32", n, seed=5)
    vals = inputs.index_payload(n)
    cfg = {"small_cutoff": 2048}
    k, v = gpu_sort_pairs(keys, vals, config=cfg)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert same_bits(gpu_sort_keys(keys, config=cfg), ek)


@pytest.mark.parametrize("case", ["all_equal", "two_values", "last_bit", "shared_prefix_u64",
                                  "extremes_i64", "max_min_u32"])
def test_degenerate_inputs(case):
    n = 300_000
    g = np.random.Generator(np.random.PCG64(77))
    if case == "all_equal":
        keys = np.full(n, 0xABCDEF01, dtype=np.uint32)
    elif case == "two_values":
        keys = np.where(g.random(n) < 0.5, 3, 0xFFFFFFF0).astype(np.uint32)
    elif case == "last_bit":
        keys = (np.uint64(0x1234567890ABCDE0) | g.integers(0, 2, size=n).astype(np.uint64))
    elif case == "shared_prefix_u64":
        keys = (np.uint64(0xFEDC000000000000) | g.integers(0, 1 << 20, size=n).astype(np.uint64))
    elif case == "extremes_i64":
        keys = g.choice(np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).max, 0, -1, 1],
                                 dtype=np.int64), size=n)
    else:
        keys = g.choice(np.array([0, 0xFFFFFFFF, 1, 0x80000000, 0x7FFFFFFF], dtype=np.uint32),
                        size=n)
    vals = inputs.index_payload(n)
    k, v = gpu_sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert same_bits(gpu_sort_keys(keys), ek)


def test_repeated_calls_reuse_workspace():
    n = 200_000
    keys = make_keys("uint64", n, seed=3)
    vals = inputs.index_payload(n)
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(n, 8, 4)
    for _ in range(3):
        tk.copy_(to_dev(keys))
        tv.copy_(to_dev(vals))
        binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)



@pytest.mark.parametrize("kind", ["u32_last_bits", "u64_last_bits", "bytes16_distinct"])
def test_equal_key_buckets_written_back(kind):
    """Buckets larger than the cutoff whose keys are all equal and that end up
    in the workspace are written back from their one key: keys that differ
    only in their last bits (after a pass-through to the first differing bit
    the next split consumes the last bits, leaving children of equal keys),
    and 16-byte keys with a few distinct values (all-equal buckets at the
    next level).  Payloads: the original index, so stability is checked."""
    n = 300_001
    g = np.random.Generator(np.random.PCG64(321))
    if kind == "u32_last_bits":
        keys = (np.uint32(0x9ABC0000) + g.choice(np.array([0, 1, 3], np.uint32), size=n)).astype(np.uint32)
        vals = inputs.index_payload(n)
    elif kind == "u64_last_bits":
        keys = (np.uint64(0x123456789AB00000) + g.choice(np.array([0, 2, 5, 7], np.uint64), size=n))
        vals = np.arange(n, dtype=np.uint64)
    else:
        base = g.integers(0, 256, size=(5, 16), dtype=np.uint8)
        keys = base[g.integers(0, 5, size=n)]
        vals = np.arange(n, dtype=np.uint64)
    k, v = gpu_sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert same_bits(gpu_sort_keys(keys), ek)
