"""Buckets already in order (the paper's early stop on a sorted sub-array):
the histogram pass records whether any adjacent pair of a bucket descends or
fails to descend; a non-decreasing bucket is finished as it stands and a
strictly decreasing one by a reversal.  Every case is compared with the
oracle's stable sort, so a wrong shortcut (a reversal of equal keys, a copy
from the wrong buffer) shows up as a mismatch."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _check_pairs(keys, vals=None, offsets=None, key_map=None):
    torch = pytest.importorskip("torch")
    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    if offsets is not None:
        binding.sort_segmented(tk, to_dev(offsets), tv, key_map=key_map)
    elif tv is None:
        binding.sort_keys(tk, key_map=key_map)
    else:
        binding.sort_pairs(tk, tv, key_map=key_map)
    torch.cuda.synchronize()
    ek = keys.copy()
    ev = None if vals is None else vals.copy()
    kw = {} if key_map is None else {"key_map": key_map}
    oracle.stable_radix(ek, ev, offsets=offsets, **kw)
    assert same_bits(to_host(tk), ek)
    if vals is not None:
        assert same_bits(to_host(tv), ev)


def _distinct_sorted(n, dtype, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    info = np.iinfo(dtype)
    x = np.unique(g.integers(0, int(info.max), size=n + n // 8, dtype=dtype, endpoint=True))
    return np.sort(x[:n]) if x.shape[0] >= n else np.sort(x)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("with_vals", [False, True])
def test_sorted_input_left_as_is(dtype, with_vals):
    require_gpu()
    keys = np.sort(inputs.uniform_keys(3 << 20, dtype, np.random.Generator(np.random.PCG64(11))))
    keys[100:200] = keys[100]              # equal runs keep their input order
    vals = inputs.index_payload(keys.shape[0]) if with_vals else None
    _check_pairs(keys, vals)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("with_vals", [False, True])
def test_strictly_decreasing_input_reversed(dtype, with_vals):
    require_gpu()
    keys = _distinct_sorted(3 << 20, dtype, 12)[::-1].copy()
    vals = inputs.index_payload(keys.shape[0]) if with_vals else None
    _check_pairs(keys, vals)


def test_decreasing_with_equal_keys_is_not_reversed():
    """Non-strictly decreasing: a reversal would break stability."""
    require_gpu()
    keys = _distinct_sorted(1 << 20, np.uint32, 13)
    keys = np.repeat(keys, 3)[::-1].copy()     # runs of three equal keys
    _check_pairs(keys, inputs.index_payload(keys.shape[0]))


def test_signed_and_float_maps_on_sorted_and_reversed_input():
    require_gpu()
    g = np.random.Generator(np.random.PCG64(14))
    f = np.sort(g.standard_normal(2 << 20).astype(np.float32))
    _check_pairs(f.copy(), inputs.index_payload(f.shape[0]), key_map=oracle.MAP_FLOAT)
    _check_pairs(np.unique(f)[::-1].copy(), None, key_map=oracle.MAP_FLOAT)
    i = np.sort(g.integers(-2**62, 2**62, size=2 << 20, dtype=np.int64))
    _check_pairs(np.unique(i)[::-1].copy(), inputs.index_payload(np.unique(i).shape[0]),
                 key_map=oracle.MAP_SIGNED)


@pytest.mark.parametrize("direction", ["ascending", "descending"])
def test_level1_buckets_in_order_inside(direction):
    """Random top byte, and inside every top-byte group the rest of the key
    runs in order with the position: level 0 splits, then every level-1 bucket
    (about 16K keys, in the workspace) is finished by a copy or a reversal."""
    require_gpu()
    n = 4 << 20
    g = np.random.Generator(np.random.PCG64(15))
    top = g.integers(0, 256, size=n, dtype=np.uint32)
    low = np.arange(n, dtype=np.uint32) * 3 + 7          # distinct, increasing
    if direction == "descending":
        low = low[::-1].copy()
    keys = (top << 24) | (low & 0x00FFFFFF)
    _check_pairs(keys, inputs.index_payload(n))
    _check_pairs(keys.copy(), None)


def test_segments_sorted_reversed_and_random():
    require_gpu()
    g = np.random.Generator(np.random.PCG64(16))
    parts, sizes = [], []
    for i in range(12):
        m = int(g.integers(9000, 60000))
        x = _distinct_sorted(m, np.uint32, 100 + i)
        kind = i % 3
        if kind == 1:
            x = x[::-1].copy()
        elif kind == 2:
            x = g.permutation(x)
        parts.append(x)
        sizes.append(x.shape[0])
    keys = np.concatenate(parts)
    off = inputs.offsets_from_sizes(np.array(sizes, dtype=np.int64))
    vals = inputs.segment_index_payload(off)
    _check_pairs(keys, vals, offsets=off)
