"""GPU parity for keys past 16 bytes and for byte strings of different
lengths (window levels over the 16-byte sort), against the oracle: the
string order of oracle.sort_strings (a proper prefix first, ties in input
order), and binar sort / stable radix sort for fixed-width wide keys."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def gpu_order(data, off, max_len=None, config=None):
    torch = pytest.importorskip("torch")
    n = len(off) - 1
    ws = torch.empty(max(binding.strings_workspace_bytes(n), 16), dtype=torch.uint8, device="cuda")
    d = to_dev(data) if len(data) else torch.zeros(1, dtype=torch.uint8, device="cuda")
    order = binding.sort_strings(d, to_dev(off), max_len=max_len, ws=ws, config=config)
    binding.check_status(ws)
    return to_host(order).view(np.uint32)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 70001, 400003])
@pytest.mark.parametrize("alphabet,max_len,prefix", [(256, 64, 0), (2, 40, 0), (4, 31, 20),
                                                     (256, 15, 0), (3, 100, 47), (256, 0, 0)])
def test_strings_against_the_oracle(n, alphabet, max_len, prefix):
    data, off = inputs.strings(n, max_len=max_len, alphabet=alphabet, shared_prefix=prefix,
                               variant=n % 7)
    assert np.array_equal(gpu_order(data, off, max_len=max_len), oracle.sort_strings(data, off))


def test_strings_duplicates_prefixes_and_empty():
    """Many copies of a few strings that are prefixes of one another (and
    empty strings): ties must keep their input order."""
    base = [b"", b"a", b"ab", b"ab\x00", b"abc", b"a" * 15, b"a" * 16, b"a" * 30, b"a" * 31,
            b"\xff" * 45, b"\x00" * 45]
    g = np.random.Generator(np.random.PCG64(8))
    pick = g.integers(0, len(base), size=200001)
    items = [base[i] for i in pick]
    off = np.concatenate([[0], np.cumsum([len(x) for x in items])]).astype(np.int64)
    data = np.frombuffer(b"".join(items), dtype=np.uint8).copy()
    assert np.array_equal(gpu_order(data, off, max_len=45), oracle.sort_strings(data, off))


def test_strings_with_the_smallest_cutoff_and_small_k():
    data, off = inputs.strings(300001, max_len=50, alphabet=3, shared_prefix=10, variant=3)
    cfg = {"small_cutoff": 2048, "bits_per_pass": 5}
    assert np.array_equal(gpu_order(data, off, max_len=50, config=cfg),
                          oracle.sort_strings(data, off))


def test_string_longer_than_max_len_is_reported():
    torch = pytest.importorskip("torch")
    data, off = inputs.strings(1000, max_len=40, min_len=35)
    n = 1000
    ws = torch.empty(binding.strings_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    binding.sort_strings(to_dev(data), to_dev(off), max_len=20, ws=ws)
    assert binding.workspace_status(ws) == binding.ERR_INVALID_ARG
    binding.sort_strings(to_dev(data), to_dev(off), max_len=40, ws=ws)     # next call is clean
    assert binding.workspace_status(ws) == binding.OK


def test_two_million_strings_by_properties():
    """At 2M strings the result is checked as a permutation whose sampled
    adjacent pairs are in order (ties: indices increasing)."""
    n = 2_000_000
    data, off = inputs.strings(n, max_len=48, alphabet=5, shared_prefix=16, variant=9)
    order = gpu_order(data, off, max_len=48).astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(n))
    g = np.random.Generator(np.random.PCG64(2))
    for k in g.integers(0, n - 1, size=20000):
        a, b = order[k], order[k + 1]
        sa, sb = bytes(data[off[a]:off[a + 1]]), bytes(data[off[b]:off[b + 1]])
        assert sa < sb or (sa == sb and a < b)


def _wide_keys(kb, n, seed):
    k = inputs.wide_keys(n, kb, shared_prefix=kb // 2, variant=seed)
    if n > 8:
        k[::3] = k[1]
        k[1::7, kb // 2:] = 0
    return k


def _expect_wide(keys, vals):
    """Stable order of fixed-width byte-string keys: the oracle's binar sort
    and stable radix sort on small cases, its string order (pinned against
    both on wide keys) on large ones."""
    n, kb = keys.shape
    if n * kb <= 3000 * 32:
        ek = keys.copy()
        oracle.binar_sort(ek, key_map=oracle.MAP_BYTES_BE)
        sk, sv = keys.copy(), vals.copy()
        oracle.stable_radix(sk, sv, key_map=oracle.MAP_BYTES_BE)
        assert same_bits(ek, sk)
        return sk, sv
    order = oracle.sort_strings(keys.reshape(-1), np.arange(n + 1, dtype=np.int64) * kb)
    return keys[order], vals[order]


@pytest.mark.parametrize("kb", [17, 32, 64, 100, 256])
@pytest.mark.parametrize("n", [1, 2, 3000, 70001])
def test_wide_byte_string_keys(kb, n):
    keys = _wide_keys(kb, n, kb + n)
    t = to_dev(keys)
    ws = binding.workspace(n, kb, 0)
    binding.sort_keys(t, ws=ws)
    binding.check_status(ws)
    for vdt in (np.uint32, np.uint64):
        vals = np.arange(n, dtype=vdt)
        ek, ev = _expect_wide(keys, vals)
        assert same_bits(to_host(t), ek)
        tk, tv = to_dev(keys), to_dev(vals)
        ws = binding.workspace(n, kb, vals.itemsize)
        binding.sort_pairs(tk, tv, ws=ws)
        binding.check_status(ws)
        assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)


@pytest.mark.parametrize("kb", [24, 32])
@pytest.mark.parametrize("key_map", [oracle.MAP_UNSIGNED, oracle.MAP_SIGNED])
def test_wide_integer_keys(kb, key_map):
    n = 50001
    g = np.random.Generator(np.random.PCG64(kb + key_map))
    keys = g.integers(0, 256, size=(n, kb), dtype=np.uint8)
    keys[::3, kb // 2:] = 0
    keys[1::5, kb // 2:] = 0xFF
    keys[::11] = keys[4]
    vals = np.arange(n, dtype=np.uint32)
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(n, kb, 4)
    binding.sort_pairs(tk, tv, key_map=key_map, ws=ws)
    binding.check_status(ws)
    sk, sv = keys.copy(), vals.copy()
    oracle.stable_radix(sk, sv, key_map=key_map)
    assert same_bits(to_host(tk), sk) and same_bits(to_host(tv), sv)
