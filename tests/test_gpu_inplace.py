"""GPU parity of the in-place, unstable mode (binar_sort_inplace): the
paper's one-bit exchange passes inside the caller's arrays.  Keys must equal
the oracle's binar sort bit for bit; the record order among equal keys is
not unique (the mode is unstable, like the paper's algorithm), so payloads
(the original index) are checked to be a permutation whose every entry
points at the key it travels with."""
import numpy as np
import pytest

import oracle
from gpu_util import expect_keys, key_map_of, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _keys(kind, n, seed):
    g = np.random.Generator(np.random.PCG64(700 + seed))
    if kind == "bytes16":
        k = g.integers(0, 256, size=(n, 16), dtype=np.uint8)
        if n > 4:
            k[::3, :10] = k[0, :10]
        return k
    if kind == "f32":
        return inputs.config3_f32(n)
    k = inputs.uniform_keys(n, np.dtype(kind), g)
    if n > 4:
        k[::5] = k[1]
    return k


def _run(keys, vals=None, config=None):
    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    kb = binding.key_layout(tk)[1]
    torch = pytest.importorskip("torch")
    ws = torch.empty(max(binding.inplace_workspace_bytes(tk.shape[0], kb,
                                                         0 if vals is None else vals.itemsize,
                                                         config), 16),
                     dtype=torch.uint8, device="cuda")
    binding.sort_inplace(tk, tv, key_map=key_map_of(keys), ws=ws, config=config)
    binding.check_status(ws)
    return to_host(tk), (None if tv is None else to_host(tv))


def _check_records(keys, k, v):
    idx = v.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(len(keys)))
    assert same_bits(keys[idx], k)


@pytest.mark.parametrize("kind", ["uint32", "uint64", "int32", "int64", "f32", "bytes16"])
@pytest.mark.parametrize("n", [0, 1, 2, 2049, 8193, 70001, 400003])
def test_inplace_keys_and_records(kind, n):
    keys = _keys(kind, n, n)
    k, _ = _run(keys)
    ek = expect_keys(keys)
    assert same_bits(k, ek)
    if n:
        vals = np.arange(n, dtype=np.uint32)
        k2, v2 = _run(keys, vals)
        assert same_bits(k2, ek)
        _check_records(keys, k2, v2)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "distinct8", "sorted", "reverse"])
def test_inplace_distributions(dtype, dist):
    n = 1_500_000
    keys = inputs.config2_keys(n, dtype, dist)
    vals = inputs.index_payload(n)
    k, v = _run(keys, vals)
    assert same_bits(k, expect_keys(keys))
    _check_records(keys, k, v)


def test_inplace_small_cutoff_and_degenerate():
    n = 3_000_001
    g = np.random.Generator(np.random.PCG64(3))
    for keys in (inputs.uniform_keys(n, np.uint32, g), np.full(n, 7, dtype=np.uint32),
                 np.where(g.random(n) < 0.5, 1, 0xFFFFFFFE).astype(np.uint32),
                 (np.uint64(0xABCD000000000000) | g.integers(0, 4, size=n).astype(np.uint64))):
        vals = np.arange(n, dtype=np.uint64)
        k, v = _run(keys, vals, config={"small_cutoff": 2048})
        assert same_bits(k, expect_keys(keys))
        _check_records(keys, k, v)


def test_inplace_full_size_and_workspace():
    """256M uint32 keys with uint32 payloads: the same keys as the stable
    out-of-place sort, records valid, and a workspace well under a quarter
    of the out-of-place one (which holds a second key and payload array)."""
    torch = pytest.importorskip("torch")
    n = 256 << 20
    assert binding.inplace_workspace_bytes(n, 4, 4) * 4 < binding.workspace_bytes(n, 4, 4)
    keys = inputs.config2_keys(n, np.uint32, "uniform")
    k0 = to_dev(keys)
    k, v = k0.clone(), torch.arange(n, dtype=torch.int32, device="cuda")
    binding.sort_inplace(k, v)
    ref = k0.clone()
    binding.sort_keys(ref)
    assert torch.equal(k, ref)
    vv = v.to(torch.int64)
    assert bool((torch.bincount(vv, minlength=n) == 1).all())
    assert torch.equal(k0.to(torch.int64)[vv], k.to(torch.int64))   # uint32 has no CUDA gather
