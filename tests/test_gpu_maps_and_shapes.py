"""GPU parity for every key map and shape the C ABI accepts.

Beyond the default maps of each dtype (covered in test_gpu_sort.py), the
header promises 16-byte keys as little-endian 128-bit unsigned and two's
complement integers, big-endian byte strings of 4 and 8 bytes, and segmented
sorts of every key width with 4- and 8-byte payloads.  Each is compared, bit
for bit, with the oracle: keys with the paper's binar sort, records with the
stable binary radix sort, one pass with the oracle's partition pass.
"""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 2049, 8193, 70001, 400003]


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _keys(kind, n, seed):
    g = np.random.Generator(np.random.PCG64(9000 + seed))
    if kind == "b16":
        k = g.integers(0, 256, size=(n, 16), dtype=np.uint8)
        if n > 8:
            k[::4, 8:] = 0                 # share the high half (little-endian) with others
            k[::3] = k[1]                  # equal keys: stability is visible
        return k
    k = inputs.uniform_keys(n, np.dtype(kind), g)
    if n > 8:
        k[::3] = k[1]
    return k


def _sort_keys(keys, key_map):
    t = to_dev(keys)
    ws = binding.workspace(t.shape[0], binding.key_layout(t)[1], 0)
    binding.sort_keys(t, key_map=key_map, ws=ws)
    binding.check_status(ws)
    return to_host(t)


def _sort_pairs(keys, vals, key_map):
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(tk.shape[0], binding.key_layout(tk)[1], tv.element_size())
    binding.sort_pairs(tk, tv, key_map=key_map, ws=ws)
    binding.check_status(ws)
    return to_host(tk), to_host(tv)


@pytest.mark.parametrize("kind,key_map", [("b16", oracle.MAP_UNSIGNED), ("b16", oracle.MAP_SIGNED),
                                          ("uint32", oracle.MAP_BYTES_BE),
                                          ("uint64", oracle.MAP_BYTES_BE)])
@pytest.mark.parametrize("n", SIZES)
def test_non_default_maps_keys_and_pairs(kind, key_map, n):
    keys = _keys(kind, n, n + key_map)
    ek = keys.copy()
    oracle.binar_sort(ek, key_map=key_map)
    assert same_bits(_sort_keys(keys, key_map), ek)
    if n == 0:
        return
    for vdt in (np.uint32, np.uint64):
        vals = np.arange(n, dtype=vdt)
        k, v = _sort_pairs(keys, vals, key_map)
        sk, sv = keys.copy(), vals.copy()
        oracle.stable_radix(sk, sv, key_map=key_map)
        assert same_bits(k, sk) and same_bits(v, sv)


def test_signed_128_extremes():
    """Two's complement 128-bit order: the minimum, -1, 0, 1 and the maximum."""
    lo = np.zeros(16, dtype=np.uint8)
    lo[15] = 0x80                                     # -2^127
    hi = np.full(16, 0xFF, dtype=np.uint8)
    hi[15] = 0x7F                                     # 2^127 - 1
    m1 = np.full(16, 0xFF, dtype=np.uint8)            # -1
    one = np.zeros(16, dtype=np.uint8)
    one[0] = 1
    zero = np.zeros(16, dtype=np.uint8)
    base = np.stack([hi, one, m1, lo, zero])
    g = np.random.Generator(np.random.PCG64(5))
    keys = base[g.integers(0, 5, size=50000)]
    got = _sort_keys(keys, oracle.MAP_SIGNED)
    as_int = [int.from_bytes(bytes(r), "little", signed=True) for r in got]
    assert as_int == sorted(int.from_bytes(bytes(r), "little", signed=True) for r in keys)


@pytest.mark.parametrize("kind,pos", [("b16", 0), ("b16", 63), ("b16", 120)])
@pytest.mark.parametrize("key_map", [oracle.MAP_UNSIGNED, oracle.MAP_SIGNED])
def test_partition_pass_128_bit_integers(kind, pos, key_map):
    n = 70001
    keys = _keys(kind, n, pos)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=pos, key_map=key_map)
    ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=key_map, pos=pos, k=8)
    assert same_bits(to_host(ko), ek) and same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)


@pytest.mark.parametrize("kind,pos", [("uint32", 0), ("uint32", 12), ("uint64", 0), ("uint64", 40)])
def test_partition_pass_big_endian_words(kind, pos):
    n = 70001
    keys = _keys(kind, n, pos)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=pos,
                                          key_map=oracle.MAP_BYTES_BE)
    ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=oracle.MAP_BYTES_BE, pos=pos, k=8)
    assert same_bits(to_host(ko), ek) and same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)


def _seg_keys(kind, n, seed):
    if kind == "f32":
        k = inputs.config3_f32(n)
    elif kind == "i64":
        k = inputs.config3_i64(n)
    elif kind == "b16":
        k = inputs.config3_bytes16(n, shared_prefix=(seed % 2 == 1))
    else:
        k = inputs.uniform_keys(n, np.dtype(kind), np.random.Generator(np.random.PCG64(seed)))
    if n > 8:
        k[::4] = k[2]
    return k


@pytest.mark.parametrize("kind,key_map", [("f32", oracle.MAP_FLOAT), ("i64", oracle.MAP_SIGNED),
                                          ("b16", oracle.MAP_BYTES_BE), ("b16", oracle.MAP_UNSIGNED),
                                          ("uint64", oracle.MAP_BYTES_BE),
                                          ("int32", oracle.MAP_SIGNED)])
@pytest.mark.parametrize("vdt", [None, np.uint32, np.uint64])
def test_segmented_every_width_and_payload(kind, key_map, vdt):
    sizes = [0, 1, 5, 2048, 2049, 9000, 0, 70001, 3, 130000, 1]
    off = inputs.offsets_from_sizes(np.asarray(sizes, dtype=np.int64))
    n = int(off[-1])
    keys = _seg_keys(kind, n, len(kind) + key_map)
    vals = None if vdt is None else inputs.segment_index_payload(off).astype(vdt)
    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    kb = binding.key_layout(tk)[1]
    ws = binding.workspace(n, kb, 0 if vals is None else vals.itemsize, len(sizes))
    binding.sort_segmented(tk, to_dev(off), tv, key_map=key_map, ws=ws)
    binding.check_status(ws)
    if vals is None:
        ek = keys.copy()
        oracle.binar_sort(ek, key_map=key_map, offsets=off)
        assert same_bits(to_host(tk), ek)
    else:
        ek, ev = keys.copy(), vals.copy()
        oracle.stable_radix(ek, ev, key_map=key_map, offsets=off)
        assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)
