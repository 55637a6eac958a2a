"""binar_partition_pass_noalloc: the partition pass for callers that cannot
allocate (their device memory is one fixed pool, or they must not trigger a
cudaMalloc); its scratch is a fixed array inside the library.

Called through the C ABI and checked, bit for bit, against the ordinary
binar_partition_pass (which takes a workspace) and against the oracle's
partition pass, on two calls in a row; then at every documented size limit
(which must succeed) and one key past it (which must be refused), always on
real device buffers of the size passed; and a look-back wait made to run out
(a tile that never publishes, through the test hook) is reported by the
status query and leaves the next call clean.  Kept in a file of its own that
pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

# (key bytes, payload bytes, map, largest n the 4 MiB scratch holds)
LIMITS = [(4, 0, oracle.MAP_UNSIGNED, 29_173_759), (4, 4, oracle.MAP_SIGNED, 25_006_079),
          (8, 4, oracle.MAP_UNSIGNED, 16_670_719), (16, 8, oracle.MAP_BYTES_BE, 8_335_359)]


def _lib():
    lib = binding.load()
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.binar_partition_pass_noalloc.argtypes = [p, p, p, p, i64, i32, i32, i32, i32, i32, p, p]
    lib.binar_partition_pass_noalloc.restype = i32
    lib.binar_partition_pass_noalloc_status.argtypes = [p, ctypes.POINTER(i32)]
    lib.binar_partition_pass_noalloc_status.restype = i32
    lib.binar_partition_pass_noalloc_debug.argtypes = [i32, i64]
    lib.binar_partition_pass_noalloc_debug.restype = i32
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    torch = pytest.importorskip("torch")
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc_pass(lib, keys, vals, pos, key_map, n=None):
    """Runs the pass on the first n records of the device tensors (all by
    default); returns (rc, keys_out, vals_out, offsets)."""
    torch = pytest.importorskip("torch")
    n = keys.shape[0] if n is None else n
    kb = binding.key_layout(keys)[1]
    vb = 0 if vals is None else vals.element_size()
    ko = torch.empty_like(keys)
    vo = None if vals is None else torch.empty_like(vals)
    offs = torch.empty(257, dtype=torch.int64, device=keys.device)
    rc = lib.binar_partition_pass_noalloc(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, kb,
                                          key_map, vb, pos, 8, _ptr(offs), _stream())
    return rc, ko, vo, offs


def _status(lib):
    st = ctypes.c_int(-1)
    assert lib.binar_partition_pass_noalloc_status(_stream(), ctypes.byref(st)) == binding.OK
    return st.value


def _keys(kb, n, g, key_map):
    if kb == 16:
        return g.integers(0, 256, size=(n, 16), dtype=np.uint8)
    dt = {(4, oracle.MAP_SIGNED): np.int32}.get((kb, key_map), np.uint32 if kb == 4 else np.uint64)
    return inputs.uniform_keys(n, dt, g)


def _vals(vb, n):
    if vb == 0:
        return None
    return np.arange(n, dtype=np.uint32 if vb == 4 else np.uint64)


def test_noalloc_pass_matches_the_workspace_pass_and_the_oracle_twice():
    require_gpu()
    lib = _lib()
    g = np.random.Generator(np.random.PCG64(4242))
    cases = [(4, 4, oracle.MAP_UNSIGNED, 3_000_017, 0), (8, 0, oracle.MAP_UNSIGNED, 1_000_003, 7),
             (16, 8, oracle.MAP_BYTES_BE, 500_001, 100), (4, 0, oracle.MAP_FLOAT, 70_001, 0)]
    for kb, vb, kmap, n, pos in cases:           # two calls in a row, the second on new data
        keys = _keys(kb, n, g, kmap) if kmap != oracle.MAP_FLOAT else inputs.config3_f32(n)
        vals = _vals(vb, n)
        tk = to_dev(keys)
        tv = None if vals is None else to_dev(vals)
        rc, ko, vo, offs = _noalloc_pass(lib, tk, tv, pos, kmap)
        assert rc == binding.OK, binding.status_string(rc)
        assert _status(lib) == binding.OK
        ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=kmap, pos=pos, k=8)
        assert same_bits(to_host(ko), ek)
        assert np.array_equal(to_host(offs), eoffs)
        if vals is not None:
            assert same_bits(to_host(vo), ev)
        wk, wv, woffs = binding.partition_pass(tk, tv, pos=pos, key_map=kmap)
        assert same_bits(to_host(ko), to_host(wk))
        assert np.array_equal(to_host(offs), to_host(woffs))
        if vals is not None:
            assert same_bits(to_host(vo), to_host(wv))


@pytest.mark.parametrize("kb,vb,kmap,limit", LIMITS)
def test_noalloc_pass_at_its_documented_limit(kb, vb, kmap, limit):
    """n = limit succeeds and matches the oracle; n = limit + 1, on buffers
    that really hold limit + 1 records, is refused before any work."""
    require_gpu()
    lib = _lib()
    g = np.random.Generator(np.random.PCG64(limit))
    keys = _keys(kb, limit + 1, g, kmap)
    vals = _vals(vb, limit + 1)
    tk = to_dev(keys)
    tv = None if vals is None else to_dev(vals)
    rc, *_ = _noalloc_pass(lib, tk, tv, 0, kmap)
    assert rc == binding.ERR_WORKSPACE_TOO_SMALL
    pos = 3
    rc, ko, vo, offs = _noalloc_pass(lib, tk, tv, pos, kmap, n=limit)
    assert rc == binding.OK, binding.status_string(rc)
    assert _status(lib) == binding.OK
    ek, ev, eoffs = oracle.partition_pass(keys[:limit], None if vals is None else vals[:limit],
                                          key_map=kmap, pos=pos, k=8)
    assert np.array_equal(to_host(offs), eoffs)
    assert same_bits(to_host(ko)[:limit], ek)
    if vals is not None:
        assert same_bits(to_host(vo)[:limit], ev)


def test_noalloc_status_reports_a_timeout_and_the_next_call_is_clean():
    require_gpu()
    lib = _lib()
    n = 6144 * 40 + 17                       # 41 tiles of the pass; tile 3 never publishes
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(77)))
    vals = _vals(4, n)
    tk, tv = to_dev(keys), to_dev(vals)
    assert lib.binar_partition_pass_noalloc_debug(4, 1_000_000) == binding.OK
    try:
        rc, *_ = _noalloc_pass(lib, tk, tv, 0, oracle.MAP_UNSIGNED)
        assert rc == binding.OK
        assert _status(lib) == binding.ERR_DEVICE_TIMEOUT
    finally:
        assert lib.binar_partition_pass_noalloc_debug(0, 0) == binding.OK
    assert _status(lib) == binding.OK        # the query cleared the word
    rc, ko, vo, offs = _noalloc_pass(lib, tk, tv, 8, oracle.MAP_UNSIGNED)
    assert rc == binding.OK
    assert _status(lib) == binding.OK
    ek, ev, eoffs = oracle.partition_pass(keys, vals, key_map=oracle.MAP_UNSIGNED, pos=8, k=8)
    assert same_bits(to_host(ko), ek) and same_bits(to_host(vo), ev)
    assert np.array_equal(to_host(offs), eoffs)
