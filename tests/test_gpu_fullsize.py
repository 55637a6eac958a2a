"""Full-size sorts in the configuration bench.py times (256M uint32 keys and
128M uint64 keys with uint32 payloads equal to the original index), the other
configurations at their full sizes, and the largest sizes: 1G records and the
largest array the C ABI accepts (2^31 - 2 records, 8 GiB per array).

At these sizes the oracle cannot recompute the output, so the checks are
properties that together fix the unique stable sort, whatever the size:
  * the keys are nondecreasing,
  * the payloads are a permutation of 0 .. n-1 (bincount == 1),
  * every output key is the input key its payload points to,
  * equal keys keep their input order (payloads increase within a run).
"""
import numpy as np
import pytest

from gpu_util import require_gpu
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _check_stable_sort(torch, keys_in, keys_out, vals_out, signed=False):
    if keys_out.dtype == torch.uint64:
        k = keys_out.view(torch.int64)
        orig = keys_in.view(torch.int64)
        # compare as unsigned: flip the sign bit
        flip = torch.tensor(-(2 ** 63), dtype=torch.int64, device=k.device)
        k = k ^ flip
        orig = orig ^ flip
    else:
        k = keys_out.to(torch.int64)
        orig = keys_in.to(torch.int64)
    v = vals_out.to(torch.int64)
    assert bool((k[1:] >= k[:-1]).all()), "keys not sorted"
    assert bool((torch.bincount(v, minlength=k.shape[0]) == 1).all()), "payload not a permutation"
    assert bool((orig[v] == k).all()), "key / payload mismatch"
    eq = k[1:] == k[:-1]
    assert bool((v[1:][eq] > v[:-1][eq]).all()), "equal keys out of input order"


@pytest.mark.parametrize("dtype,n,dist", [
    (np.uint32, 256 << 20, "uniform"),
    (np.uint64, 128 << 20, "uniform"),
    (np.uint32, 256 << 20, "sorted"),
    (np.uint32, 256 << 20, "reverse"),
    (np.uint32, 32 << 20, "zipf"),
    (np.uint32, 64 << 20, "distinct8"),
])
def test_full_size_pairs(dtype, n, dist):
    require_gpu()
    torch = pytest.importorskip("torch")
    keys = inputs.config2_keys(n, dtype, dist)
    vals = inputs.index_payload(n)
    k0 = torch.from_numpy(keys).cuda()
    tk = k0.clone()
    tv = torch.from_numpy(vals).cuda()
    del keys, vals
    ws = binding.workspace(n, np.dtype(dtype).itemsize, 4)
    binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)
    _check_stable_sort(torch, k0, tk, tv)


def test_full_size_keys_only_uniform_u32():
    require_gpu()
    torch = pytest.importorskip("torch")
    n = 256 << 20
    keys = inputs.config2_keys(n, np.uint32, "uniform")
    k0 = torch.from_numpy(keys).cuda()
    tk = k0.clone()
    ws = binding.workspace(n, 4, 0)
    binding.sort_keys(tk, ws=ws)
    binding.check_status(ws)
    k = tk.to(torch.int64)
    assert bool((k[1:] >= k[:-1]).all())
    # same multiset: both sorted copies agree with a library sort of the input
    ref = torch.sort(k0.to(torch.int64)).values
    assert bool((ref == k).all())


def _check_stable_by_order_key(torch, okey_in, okey_out, vals_out, eq_out=None):
    """okey_*: int64 tensors (or tuples of them, compared lexicographically) whose
    order is the key order; checks the stable-sort properties of the output."""
    if not isinstance(okey_out, tuple):
        okey_in, okey_out = (okey_in,), (okey_out,)
    v = vals_out.to(torch.int64)
    n = v.shape[0]
    assert bool((torch.bincount(v, minlength=n) == 1).all()), "payload not a permutation"
    for a, b in zip(okey_in, okey_out):
        assert bool((a[v] == b).all()), "key / payload mismatch"
    # nondecreasing, lexicographically
    less = torch.zeros(n - 1, dtype=torch.bool, device=v.device)
    equal = torch.ones(n - 1, dtype=torch.bool, device=v.device)
    for b in okey_out:
        less |= equal & (b[:-1] < b[1:])
        equal &= b[:-1] == b[1:]
    assert bool((less | equal).all()), "keys not sorted"
    assert bool((v[1:][equal] > v[:-1][equal]).all()), "equal keys out of input order"


def test_full_size_config3_float32_pairs():
    """64M float32 (normal mixed with +-0, +-inf, denormals, duplicates)."""
    require_gpu()
    torch = pytest.importorskip("torch")
    n = 64 << 20
    keys = inputs.config3_f32(n)
    k0 = torch.from_numpy(keys).cuda()
    tk, tv = k0.clone(), torch.from_numpy(inputs.index_payload(n)).cuda()
    ws = binding.workspace(n, 4, 4)
    binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)

    def order(t):   # IEEE order of the bit patterns (-0 < +0, NaNs by sign)
        u = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        return torch.where(u >= 2 ** 31, (~u) & 0xFFFFFFFF, u | 2 ** 31)
    _check_stable_by_order_key(torch, order(k0), order(tk), tv)


def test_full_size_config3_int64_pairs():
    require_gpu()
    torch = pytest.importorskip("torch")
    n = 64 << 20
    k0 = torch.from_numpy(inputs.config3_i64(n)).cuda()
    tk, tv = k0.clone(), torch.from_numpy(inputs.index_payload(n)).cuda()
    ws = binding.workspace(n, 8, 4)
    binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)
    _check_stable_by_order_key(torch, k0, tk, tv)


@pytest.mark.parametrize("shared_prefix", [False, True])
def test_full_size_config3_bytes16_pairs(shared_prefix):
    """16M 16-byte strings in memcmp order (uniform bytes, or a shared 12-byte prefix)."""
    require_gpu()
    torch = pytest.importorskip("torch")
    n = 16 << 20
    k0 = torch.from_numpy(inputs.config3_bytes16(n, shared_prefix=shared_prefix)).cuda()
    tk, tv = k0.clone(), torch.from_numpy(inputs.index_payload(n)).cuda()
    ws = binding.workspace(n, 16, 4)
    binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)

    def order(t):   # big-endian halves, as signed int64 with the sign bit flipped
        b = t.to(torch.int64)
        hi = torch.zeros(t.shape[0], dtype=torch.int64, device=t.device)
        lo = torch.zeros_like(hi)
        for i in range(8):
            hi = (hi << 8) | b[:, i]
            lo = (lo << 8) | b[:, 8 + i]
        flip = torch.tensor(-(2 ** 63), dtype=torch.int64, device=t.device)
        return hi ^ flip, lo ^ flip
    _check_stable_by_order_key(torch, order(k0), order(tk), tv)


@pytest.mark.parametrize("dtype,n", [
    (np.uint32, 1 << 30),                       # 1G records: the top of the benchmark's size range
    (np.uint64, 1 << 30),                       # 8 GiB of keys
    (np.uint32, binding.MAX_BUCKET_KEYS),       # the largest array the C ABI accepts
])
def test_largest_sizes_pairs(dtype, n):
    """Arrays of 4 to 16 GiB: every byte offset beyond 4 GiB, tile and job
    counts near the workspace bounds and, for 2^31 - 2 uniform 4-byte keys, a
    third partition level (level-2 buckets of about 32K keys).  Keys come
    from the device generator, payloads are the input positions."""
    require_gpu()
    torch = pytest.importorskip("torch")
    tdt = torch.uint32 if dtype == np.uint32 else torch.uint64
    k0 = torch.empty(n, dtype=tdt, device="cuda")
    binding.generate(k0, 0x0811_3448 + n)
    tk = k0.clone()
    tv = torch.arange(n, dtype=torch.int32, device="cuda")
    ws = binding.workspace(n, np.dtype(dtype).itemsize, 4)
    binding.sort_pairs(tk, tv, ws=ws)
    binding.check_status(ws)
    del ws
    _check_stable_sort(torch, k0, tk, tv)
    del k0, tk, tv
    torch.cuda.empty_cache()


def test_billion_keys_only_u32():
    require_gpu()
    torch = pytest.importorskip("torch")
    n = 1 << 30
    k0 = torch.empty(n, dtype=torch.uint32, device="cuda")
    binding.generate(k0, 0x3448_0811)
    tk = k0.clone()
    ws = binding.workspace(n, 4, 0)
    binding.sort_keys(tk, ws=ws)
    binding.check_status(ws)
    del ws
    k = tk.to(torch.int64)
    del tk
    ref = torch.sort(k0.to(torch.int64)).values
    assert bool((ref == k).all())
    del k0, k, ref
    torch.cuda.empty_cache()
