"""binar_partition_pass_noalloc: the partition pass for callers that cannot
allocate (their device memory is one fixed pool, or they must not trigger a
cudaMalloc); its scratch is a fixed array inside the library.

Called through the C ABI and checked, bit for bit, against the ordinary
binar_partition_pass (which takes a workspace) on two calls in a row.  Kept
in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import require_gpu, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    lib = binding.load()
    fn = lib.binar_partition_pass_noalloc
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    fn.argtypes = [p, p, p, p, i64, i32, i32, i32, i32, i32, p, p]
    fn.restype = i32
    return fn


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc_pass(fn, keys, vals, pos, key_map):
    torch = pytest.importorskip("torch")
    n, kb, _ = binding.key_layout(keys)
    vb = 0 if vals is None else vals.element_size()
    ko = torch.empty_like(keys)
    vo = None if vals is None else torch.empty_like(vals)
    offs = torch.empty(257, dtype=torch.int64, device=keys.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, kb, key_map, vb, pos, 8, _ptr(offs),
            stream)
    assert rc == binding.OK, binding.status_string(rc)
    return ko, vo, offs


def test_noalloc_pass_matches_the_workspace_pass_twice():
    require_gpu()
    fn = _noalloc_fn()
    g = np.random.Generator(np.random.PCG64(4242))
    cases = [
        (inputs.uniform_keys(3_000_017, np.uint32, g), np.arange(3_000_017, dtype=np.uint32), 0,
         binding.MAP_UNSIGNED),
        (inputs.uniform_keys(1_000_003, np.uint64, g), None, 7, binding.MAP_UNSIGNED),
    ]
    for keys, vals, pos, kmap in cases:          # two calls in a row
        tk = to_dev(keys)
        tv = None if vals is None else to_dev(vals)
        ko, vo, offs = _noalloc_pass(fn, tk, tv, pos, kmap)
        ek, ev, eoffs = binding.partition_pass(tk, tv, pos=pos, key_map=kmap)
        assert np.array_equal(to_host(ko).view(np.uint8), to_host(ek).view(np.uint8))
        assert np.array_equal(to_host(offs), to_host(eoffs))
        if vals is not None:
            assert np.array_equal(to_host(vo), to_host(ev))


def test_noalloc_pass_rejects_sizes_beyond_its_scratch():
    require_gpu()
    fn = _noalloc_fn()
    fake = ctypes.c_void_p(0x1000)
    rc = fn(fake, None, fake, None, 40_000_000, 4, binding.MAP_UNSIGNED, 0, 0, 8, None, None)
    assert rc == binding.ERR_WORKSPACE_TOO_SMALL
