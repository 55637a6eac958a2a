"""GPU parity for one partition pass and for segmented sorts."""
import numpy as np
import pytest

import oracle
from gpu_util import expect_pairs, key_map_of, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("kind,pos", [("uint32", 0), ("uint32", 8), ("uint32", 24), ("uint32", 29),
                                      ("uint64", 5), ("uint64", 56), ("int64", 0), ("f32", 0),
                                      ("bytes16", 0), ("bytes16", 100)])
@pytest.mark.parametrize("n", [1, 1000, 8192, 8193, 333333])
def test_partition_pass_against_oracle(kind, pos, n):
    g = np.random.Generator(np.random.PCG64(n + pos))
    if kind == "bytes16":
        keys = g.integers(0, 256, size=(n, 16), dtype=np.uint8)
    elif kind == "f32":
        keys = inputs.config3_f32(n)
    else:
        keys = inputs.uniform_keys(n, np.dtype(kind), g)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=pos,
                                          key_map=key_map_of(keys))
    ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=key_map_of(keys), pos=pos, k=8)
    assert same_bits(to_host(ko), ek)
    assert same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)
    # keys only
    ko2, _, offs2 = binding.partition_pass(to_dev(keys), None, pos=pos, key_map=key_map_of(keys))
    assert same_bits(to_host(ko2), ek)
    assert np.array_equal(to_host(offs2), eoffs)



@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("pos", [0, 24])
@pytest.mark.parametrize("n", [6144, 12288, 18433, 61440])
def test_partition_pass_full_tiles_with_random_payloads(n, pos, tile):
    """4-byte keys with 4-byte payloads are staged as 8-byte records that fill
    the tile's key and payload buffers: sizes that are whole tiles of both
    shapes (6144 and 4096 keys: every tile full) and one key past them,
    payloads unrelated to the keys."""
    g = np.random.Generator(np.random.PCG64(7000 + n + pos))
    keys = inputs.uniform_keys(n, np.uint32, g)
    vals = inputs.uniform_keys(n, np.uint32, g)
    cfg = {"tile_keys": binding.tile_choices(4, 4)[tile]}
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=pos, config=cfg)
    ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=key_map_of(keys), pos=pos, k=8)
    assert same_bits(to_host(ko), ek)
    assert same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)

def test_partition_pass_empty():
    keys = np.zeros(0, dtype=np.uint32)
    _, _, offs = binding.partition_pass(to_dev(keys), None, pos=0)
    assert np.array_equal(to_host(offs), np.zeros(257, dtype=np.int64))


def _segmented_case(sizes, dtype=np.uint32, with_vals=True, seed=0):
    off = inputs.offsets_from_sizes(np.asarray(sizes, dtype=np.int64))
    n = int(off[-1])
    g = np.random.Generator(np.random.PCG64(500 + seed))
    keys = inputs.uniform_keys(n, dtype, g)
    if n > 10:
        keys[::3] = keys[1]
    vals = inputs.segment_index_payload(off) if with_vals else None
    tk = to_dev(keys)
    tv = to_dev(vals) if with_vals else None
    toff = to_dev(off)
    ws = binding.workspace(n, np.dtype(dtype).itemsize, 4 if with_vals else 0, len(sizes))
    binding.sort_segmented(tk, toff, tv, ws=ws)
    binding.check_status(ws)
    if with_vals:
        ek, ev = expect_pairs(keys, vals, offsets=off)
        assert same_bits(to_host(tk), ek)
        assert same_bits(to_host(tv), ev)
    else:
        ek = keys.copy()
        oracle.binar_sort(ek, key_map=key_map_of(keys), offsets=off)
        assert same_bits(to_host(tk), ek)


def test_segmented_edge_segments():
    C = 8192
    sizes = [0, 1, 2, 0, 5, C - 1, C, C + 1, 3 * C + 7, 1, 0, 100000, 17]
    _segmented_case(sizes)
    _segmented_case(sizes, with_vals=False, seed=1)
    _segmented_case(sizes, dtype=np.uint64, seed=2)


def test_segmented_config4_recipe_small():
    """Config 4 recipe (log-uniform sizes) scaled to 4M keys in 3000 segments."""
    sizes = inputs.config4_segment_sizes(total=4 << 20, count=3000)
    _segmented_case(sizes, seed=3)


def test_segmented_single_segment_equals_pairs_sort():
    n = 250_000
    _segmented_case([n], seed=4)


def test_segmented_rejects_bad_offsets():
    keys = to_dev(np.arange(100, dtype=np.uint32)[::-1].copy())
    off = to_dev(np.array([0, 50, 40, 100], dtype=np.int64))   # decreasing pair
    ws = binding.workspace(100, 4, 0, 3)
    binding.sort_segmented(keys, off, None, ws=ws)
    assert binding.workspace_status(ws) == binding.ERR_INVALID_ARG
