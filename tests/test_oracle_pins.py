"""Pins the CPU oracle to facts fixed by the paper and by mathematics.

Every check compares the oracle against something other than itself: brute
force over all small inputs, library sorts (numpy) on the encoded keys,
closed forms of the encodings (IEEE-754 and two's complement order), the
complexity bound of the time analysis (at most one visit per element per bit),
and invariants of a partition pass.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import MAP_BYTES_BE, MAP_FLOAT, MAP_SIGNED, MAP_UNSIGNED
from paper_0811_3448_gb300 import inputs


def _rows_offsets(rows, length):
    return np.arange(rows + 1, dtype=np.int64) * length


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("length", [0, 1, 2, 3, 4, 5])
def test_exhaustive_nybble_arrays(length):
    """Every array of `length` nybbles (16^length arrays) sorts like np.sort."""
    rows = 16 ** length
    if length == 0:
        keys = np.zeros(0, dtype=np.uint8)
        assert oracle.binar_sort(keys, w=4) == 0
        return
    digits = np.indices((16,) * length).reshape(length, -1).T.astype(np.uint8)
    keys = (digits << 4).astype(np.uint8).reshape(-1)
    expect = np.sort(keys.reshape(rows, length), axis=1).reshape(-1)
    visits = oracle.binar_sort(keys, w=4, offsets=_rows_offsets(rows, length))
    assert np.array_equal(keys, expect)
    assert visits <= 4 * rows * length


def test_all_permutations_with_duplicates():
    """All 8! orders of a multiset with repeats sort to the same array."""
    base = np.array([3, 1, 3, 0, 7, 1, 15, 3], dtype=np.uint8) << 4
    perms = np.array(list(itertools.permutations(range(8))), dtype=np.int64)
    keys = base[perms].astype(np.uint8).reshape(-1)
    oracle.binar_sort(keys, w=4, offsets=_rows_offsets(len(perms), 8))
    expect = np.tile(np.sort(base), len(perms))
    assert np.array_equal(keys, expect)


# --------------------------------------------------------- library cross-check
@pytest.mark.parametrize("dtype,key_map", [
    (np.uint32, MAP_UNSIGNED), (np.uint64, MAP_UNSIGNED), (np.int32, MAP_SIGNED),
    (np.int64, MAP_SIGNED), (np.uint16, MAP_UNSIGNED), (np.int8, MAP_SIGNED)])
def test_integer_keys_match_numpy(dtype, key_map):
    g = np.random.Generator(np.random.PCG64(11))
    keys = inputs.uniform_keys(20000, dtype, g)
    expect = np.sort(keys)
    visits = oracle.binar_sort(keys, key_map=key_map)
    assert np.array_equal(keys, expect)
    assert visits <= 8 * keys.dtype.itemsize * len(keys)


def test_signed_extremes():
    keys = np.array([0, -1, np.iinfo(np.int64).max, np.iinfo(np.int64).min, 1,
                     np.iinfo(np.int64).min + 1, -2], dtype=np.int64)
    expect = np.sort(keys)
    oracle.binar_sort(keys, key_map=MAP_SIGNED)
    assert np.array_equal(keys, expect)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_float_keys_total_order(dtype):
    """IEEE-754 order: -NaN < -inf < negatives < -0 < +0 < positives < +inf < +NaN."""
    g = np.random.Generator(np.random.PCG64(12))
    x = g.standard_normal(5000).astype(dtype)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -1.0], dtype=dtype)
    tiny = np.finfo(dtype).smallest_subnormal
    special = np.concatenate([special, np.array([tiny, -tiny, 3 * tiny, -7 * tiny], dtype=dtype)])
    keys = np.concatenate([x, special])
    g.shuffle(keys)
    oracle.binar_sort(keys, key_map=MAP_FLOAT)
    # values are nondecreasing and, among zeros, -0 precedes +0
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    zeros = keys[keys == 0]
    assert np.signbit(zeros[0]) and not np.signbit(zeros[-1])
    assert np.array_equal(np.sort(keys), keys)  # same multiset, numpy order on values
    # NaNs by sign: a negative NaN sorts first, a positive NaN last
    ut = np.uint32 if dtype == np.float32 else np.uint64
    sign = ut(1) << ut(8 * np.dtype(dtype).itemsize - 1)
    pnan = np.array([np.nan], dtype=dtype)
    nnan = pnan.view(ut) | sign
    k2 = np.concatenate([keys, pnan, nnan.view(dtype)])
    oracle.binar_sort(k2, key_map=MAP_FLOAT)
    assert np.isnan(k2[0]) and np.signbit(k2[0])
    assert np.isnan(k2[-1]) and not np.signbit(k2[-1])


def test_float_map_is_monotone_on_finite_values():
    g = np.random.Generator(np.random.PCG64(13))
    x = np.unique(g.standard_normal(4000).astype(np.float32) * 1e3)
    m = oracle.map_keys(x, MAP_FLOAT)
    as_int = m.astype(np.uint64) @ (np.uint64(256) ** np.arange(3, -1, -1, dtype=np.uint64))
    assert np.all(np.diff(as_int.astype(np.int64)) > 0)


def test_bytes_be_match_lexicographic():
    k = inputs.config3_bytes16(3000)
    k[::7, :12] = k[0, :12]  # shared prefixes
    expect = np.array(sorted(bytes(r) for r in k), dtype=object)
    oracle.binar_sort(k, key_map=MAP_BYTES_BE)
    assert [bytes(r) for r in k] == list(expect)


def test_unsigned_128_little_endian():
    g = np.random.Generator(np.random.PCG64(14))
    k = g.integers(0, 256, size=(2000, 16), dtype=np.uint8)
    k[::3, 8:] = 0
    as_int = [int.from_bytes(bytes(r), "little") for r in k]
    oracle.binar_sort(k, key_map=MAP_UNSIGNED)
    got = [int.from_bytes(bytes(r), "little") for r in k]
    assert got == sorted(as_int)


# ------------------------------------------------------------- complexity
def test_visits_closed_forms():
    # all keys equal: every bit is a pass-through over all n elements -> w * n
    keys = np.full(1000, 0xDEADBEEF, dtype=np.uint32)
    assert oracle.binar_sort(keys) == 32 * 1000
    # n <= 1: base case, no visits
    assert oracle.binar_sort(np.array([5], dtype=np.uint32)) == 0
    # distinct keys 0..n-1 with n = 2^b in a w-bit word: the w-b leading zero bits
    # pass through over all n, then the b low bits split into complete halves
    n, b = 1024, 10
    keys = np.arange(n, dtype=np.uint32)[::-1].copy()
    assert oracle.binar_sort(keys) == (32 - b) * n + b * n
    assert np.array_equal(keys, np.arange(n, dtype=np.uint32))


# ------------------------------------------------------------- stable order
@pytest.mark.parametrize("dtype,key_map,dist", [
    (np.uint32, MAP_UNSIGNED, "distinct8"), (np.uint32, MAP_UNSIGNED, "zipf"),
    (np.uint64, MAP_UNSIGNED, "uniform"), (np.int64, MAP_SIGNED, None),
    (np.float32, MAP_FLOAT, None)])
def test_stable_radix_matches_stable_argsort(dtype, key_map, dist):
    n = 5000
    if dist is not None:
        keys = inputs.config2_keys(n, dtype, dist)
    elif dtype == np.float32:
        keys = inputs.config3_f32(n)
    else:
        keys = inputs.config3_i64(n)
    vals = inputs.index_payload(n)
    mapped = oracle.map_keys(keys, key_map)
    # library reference: stable argsort on the encoded key bytes
    order = np.lexsort(mapped.T[::-1])  # lexsort is stable; first key column most significant
    k, v = keys.copy(), vals.copy()
    oracle.stable_radix(k, v, key_map=key_map)
    assert np.array_equal(v, vals[order])
    assert np.array_equal(k.view(np.uint8), keys[order].view(np.uint8))
    # keys agree with the paper's (unstable) binar sort
    k2 = keys.copy()
    oracle.binar_sort(k2, key_map=key_map)
    assert np.array_equal(k2.view(np.uint8), k.view(np.uint8))


def test_stable_radix_segments_and_identity_cases():
    sizes = np.array([0, 1, 2, 17, 0, 300, 5], dtype=np.int64)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(3))) % np.uint32(7)
    vals = inputs.segment_index_payload(off)
    k, v = keys.copy(), vals.copy()
    oracle.stable_radix(k, v, offsets=off)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        order = np.argsort(keys[a:b], kind="stable")
        assert np.array_equal(k[a:b], keys[a:b][order])
        assert np.array_equal(v[a:b], vals[a:b][order])
    # sorted input keeps the identity payload; all-equal input is unchanged
    ks = np.sort(inputs.uniform_keys(1000, np.uint32, np.random.Generator(np.random.PCG64(4))))
    vs = inputs.index_payload(1000)
    oracle.stable_radix(ks, vs)
    assert np.array_equal(vs, np.arange(1000, dtype=np.uint32))
    ke = np.full(100, 9, dtype=np.uint64)
    ve = inputs.index_payload(100)
    oracle.stable_radix(ke, ve)
    assert np.array_equal(ve, np.arange(100, dtype=np.uint32))


# ------------------------------------------------------------- partition pass
@pytest.mark.parametrize("dtype,key_map,pos,k", [
    (np.uint32, MAP_UNSIGNED, 0, 8), (np.uint32, MAP_UNSIGNED, 8, 8),
    (np.uint32, MAP_UNSIGNED, 28, 8), (np.uint64, MAP_UNSIGNED, 5, 11),
    (np.float32, MAP_FLOAT, 0, 8), (np.int64, MAP_SIGNED, 0, 1)])
def test_partition_pass_invariants(dtype, key_map, pos, k):
    n = 7000
    if dtype == np.float32:
        keys = inputs.config3_f32(n)
    else:
        keys = inputs.uniform_keys(n, dtype, np.random.Generator(np.random.PCG64(5)))
    vals = inputs.index_payload(n)
    ko, vo, offs = oracle.partition_pass(keys, vals, key_map=key_map, pos=pos, k=k)
    w = 8 * keys.dtype.itemsize
    mapped = oracle.map_keys(keys, key_map)
    as_int = np.zeros(n, dtype=object)
    for c in range(mapped.shape[1]):
        as_int = as_int * 256 + mapped[:, c].astype(object)
    shift = w - pos - k
    digit = np.array([(int(x) >> shift) if shift >= 0 else (int(x) << -shift) for x in as_int],
                     dtype=object)
    digit = np.array([int(d) & ((1 << k) - 1) for d in digit], dtype=np.int64)
    # library reference: stable argsort by digit
    order = np.argsort(digit, kind="stable")
    assert np.array_equal(vo, vals[order])
    assert np.array_equal(ko.view(np.uint8), keys[order].view(np.uint8))
    hist = np.bincount(digit, minlength=1 << k)
    assert np.array_equal(offs, np.concatenate([[0], np.cumsum(hist)]))
    d_out = digit[vo.astype(np.int64)]
    assert np.all(np.diff(d_out) >= 0)


# ------------------------------------------------------------- rank by definition
@pytest.mark.parametrize("dtype,key_map", [(np.uint32, MAP_UNSIGNED), (np.int64, MAP_SIGNED),
                                           (np.float32, MAP_FLOAT)])
def test_rank_of_matches_searchsorted(dtype, key_map):
    g = np.random.Generator(np.random.PCG64(21))
    if dtype == np.float32:
        keys = inputs.config3_f32(3000)
        keys = keys[~np.isnan(keys)]
    else:
        keys = inputs.uniform_keys(3000, dtype, g) % dtype(50)
    s = np.sort(keys)
    for probe in list(keys[:40]) + [dtype(7)]:
        lt, le = oracle.rank_of(keys, np.array([probe], dtype=dtype), key_map)
        if dtype == np.float32 and probe == 0:
            continue  # +0 and -0 are distinct keys here, equal for numpy
        assert lt == np.searchsorted(s, probe, side="left")
        assert le == np.searchsorted(s, probe, side="right")


def test_occurrence_finds_the_jth_copy():
    keys = np.array([5, 3, 5, 5, 1, 3], dtype=np.uint32)
    five = np.array([5], dtype=np.uint32)
    assert [oracle.occurrence(keys, five, j) for j in range(4)] == [0, 2, 3, -1]
    assert oracle.occurrence(keys, np.array([1], dtype=np.uint32), 0) == 4


# ------------------------------------------------------------- parallel variant
@pytest.mark.parametrize("dtype,key_map,dist", [
    (np.uint32, MAP_UNSIGNED, "uniform"), (np.uint32, MAP_UNSIGNED, "zipf"),
    (np.uint32, MAP_UNSIGNED, "distinct8"), (np.uint32, MAP_UNSIGNED, "sorted"),
    (np.uint64, MAP_UNSIGNED, "uniform"), (np.uint64, MAP_UNSIGNED, "reverse"),
    (np.int64, MAP_SIGNED, None), (np.float32, MAP_FLOAT, None), ("b16", MAP_BYTES_BE, None)])
@pytest.mark.parametrize("log2_groups", [0, 1, 4, 8])
def test_parallel_variant_sorts(dtype, key_map, dist, log2_groups):
    """The parallel variant ("Algorithm Variants": group p holds the elements
    whose leading bits spell p, each group sorted on its own) gives the keys of
    np.sort / sorted(bytes), carries every payload with its key, and places each
    element at most once per bit plus once for the grouping pass
    ("Performance Time Analysis": one access per bit per element)."""
    n = 6000
    if dist is not None:
        keys = inputs.config2_keys(n, dtype, dist)
    elif dtype == np.float32:
        keys = inputs.config3_f32(n)
    elif dtype == np.int64:
        keys = inputs.config3_i64(n)
    else:
        keys = inputs.config3_bytes16(n)
        keys[::5, :12] = keys[0, :12]
    vals = inputs.index_payload(n)
    k, v = keys.copy(), vals.copy()
    visits = oracle.binar_sort_parallel(k, v, key_map=key_map, log2_groups=log2_groups)
    if keys.ndim == 2:
        assert [bytes(r) for r in k] == sorted(bytes(r) for r in keys)
        assert np.array_equal(keys[v.astype(np.int64)], k)
        w = 128
    else:
        expect = np.sort(keys)
        if dtype == np.float32:   # NaN-free input; -0 and +0 compare equal in numpy
            assert np.all(k[1:] >= k[:-1])
            assert np.array_equal(np.sort(k), expect)
        else:
            assert np.array_equal(k, expect)
        assert np.array_equal(keys[v.astype(np.int64)].view(np.uint8), k.view(np.uint8))
        w = 8 * keys.dtype.itemsize
    assert np.array_equal(np.sort(v), vals)
    assert visits <= (w + 1) * n


def test_parallel_variant_agrees_with_binar_sort_on_keys():
    """Both give the unique nondecreasing arrangement, so their keys agree bit
    for bit, whatever the split width (edge cases: n = 0, 1, all equal)."""
    for n in (0, 1, 2, 257):
        for fill in (None, 7):
            keys = (np.full(n, fill, dtype=np.uint32) if fill is not None else
                    inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(n))))
            a, b = keys.copy(), keys.copy()
            oracle.binar_sort(a)
            oracle.binar_sort_parallel(b, log2_groups=3)
            assert np.array_equal(a, b)


# ------------------------------------------------------------- long and variable-length keys
def _string_list(data, off):
    return [bytes(data[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def test_strings_brute_force_all_short_binary_strings():
    """Every string over {0, 1} of length 0..5 (63 strings), each twice,
    shuffled: the order is the sorted list (a proper prefix first) and equal
    strings keep their input order."""
    words = [bytes(w) for L in range(6) for w in itertools.product((0, 1), repeat=L)]
    g = np.random.Generator(np.random.PCG64(31))
    items = words + words
    perm = g.permutation(len(items))
    items = [items[i] for i in perm]
    off = np.concatenate([[0], np.cumsum([len(w) for w in items])]).astype(np.int64)
    data = np.frombuffer(b"".join(items), dtype=np.uint8).copy()
    order = oracle.sort_strings(data, off)
    assert [items[i] for i in order] == sorted(items)
    for a, b in zip(order[:-1], order[1:]):           # stable: equal strings in input order
        if items[a] == items[b]:
            assert a < b


@pytest.mark.parametrize("alphabet,max_len,prefix", [(256, 40, 0), (3, 12, 0), (2, 70, 30),
                                                     (256, 0, 0)])
def test_strings_match_python_sorted(alphabet, max_len, prefix):
    """Python orders bytes lexicographically with a proper prefix first, and
    sorted() is stable: the library-routine reference."""
    data, off = inputs.strings(4000, max_len=max_len, alphabet=alphabet, shared_prefix=prefix)
    items = _string_list(data, off)
    order = oracle.sort_strings(data, off)
    assert list(order) == sorted(range(len(items)), key=lambda i: items[i])


def test_strings_edge_cases():
    assert len(oracle.sort_strings(np.zeros(0, np.uint8), np.zeros(1, np.int64))) == 0
    data = np.frombuffer(b"bab" + b"ba" + b"" + b"b" + b"\x00", dtype=np.uint8).copy()
    off = np.array([0, 3, 5, 5, 6, 7], dtype=np.int64)   # "bab", "ba", "", "b", "\0"
    assert list(oracle.sort_strings(data, off)) == [2, 4, 3, 1, 0]


@pytest.mark.parametrize("kb", [17, 32, 64, 100, 256])
def test_wide_byte_string_keys(kb):
    """Fixed-width keys past 16 bytes: binar sort (bit by bit over all 8*kb
    bits) gives sorted(bytes); the stable radix sort keeps equal keys in input
    order; both agree with the string order of the same bytes."""
    n = 600 if kb == 256 else 2000
    k = inputs.wide_keys(n, kb, shared_prefix=kb // 2)
    k[::4] = k[1]
    keys = k.copy()
    visits = oracle.binar_sort(keys, key_map=MAP_BYTES_BE)
    assert [bytes(r) for r in keys] == sorted(bytes(r) for r in k)
    assert visits <= 8 * kb * n
    ks, vs = k.copy(), inputs.index_payload(n)
    oracle.stable_radix(ks, vs, key_map=MAP_BYTES_BE)
    order = oracle.sort_strings(k.reshape(-1), np.arange(n + 1, dtype=np.int64) * kb)
    assert np.array_equal(vs, order)
    assert np.array_equal(ks, k[order])


@pytest.mark.parametrize("kb", [32, 48])
def test_wide_integer_keys(kb):
    """Little-endian unsigned and two's complement integers of 256 / 384 bits."""
    g = np.random.Generator(np.random.PCG64(kb))
    k = g.integers(0, 256, size=(1500, kb), dtype=np.uint8)
    k[::3, kb // 2:] = 0
    k[1::5, kb // 2:] = 0xFF
    for key_map, signed in ((MAP_UNSIGNED, False), (MAP_SIGNED, True)):
        keys = k.copy()
        oracle.binar_sort(keys, key_map=key_map)
        got = [int.from_bytes(bytes(r), "little", signed=signed) for r in keys]
        assert got == sorted(int.from_bytes(bytes(r), "little", signed=signed) for r in k)
