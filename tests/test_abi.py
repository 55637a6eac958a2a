"""The C-ABI library builds, loads and exports every symbol that
include/binar.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_0811_3448_gb300 import binding
from paper_0811_3448_gb300 import build as lib_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "binar.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(binar_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("binar_sort_keys", "binar_sort_pairs", "binar_sort_segmented",
                     "binar_workspace_bytes", "binar_workspace_status", "binar_status_string",
                     "binar_partition_pass"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (binar_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_status_strings_and_version(lib):
    assert binding.status_string(0) == "ok"
    for code in range(1, 8):
        assert binding.status_string(code) not in ("ok", "unknown status")
    assert binding.status_string(99) == "unknown status"
    assert re.match(r"\d+\.\d+\.\d+", binding.version())


def test_workspace_bytes_grows_with_n(lib):
    a = binding.workspace_bytes(1 << 20, 4, 4)
    b = binding.workspace_bytes(1 << 24, 4, 4)
    assert b > a >= (1 << 20) * 8
    assert binding.workspace_bytes(1 << 20, 16, 8) >= (1 << 20) * 24
    assert binding.workspace_bytes(0, 4, 0) > 0
    with pytest.raises(binding.BinarError):
        binding.workspace_bytes(10, 3, 0)
    with pytest.raises(binding.BinarError):
        binding.workspace_bytes(10, 4, 2)


def _call_keys(lib, keys, n, kb, kmap, ws, wsb, cfg=None):
    return lib.binar_sort_keys(keys, n, kb, kmap, ws, wsb, cfg, None)


def test_argument_checks_need_no_gpu(lib):
    aligned = ctypes.c_void_p(0x1000)
    odd = ctypes.c_void_p(0x1002)
    big = 1 << 40
    # bad key width, bad map, FLOAT on 16-byte keys
    assert _call_keys(lib, aligned, 10, 3, 0, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, aligned, 10, 4, 7, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, aligned, 10, 16, binding.MAP_FLOAT, aligned, big) == binding.ERR_UNSUPPORTED
    # misaligned or missing pointers
    assert _call_keys(lib, odd, 10, 4, 0, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, None, 10, 4, 0, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, aligned, 10, 4, 0, odd, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, ctypes.c_void_p(0x1004), 10, 8, 0, aligned, big) == binding.ERR_INVALID_ARG
    # negative n, too many keys, workspace too small
    assert _call_keys(lib, aligned, -1, 4, 0, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, aligned, binding.MAX_BUCKET_KEYS + 1, 4, 0, aligned, big) == \
        binding.ERR_UNSUPPORTED
    assert _call_keys(lib, aligned, 1000, 4, 0, aligned, 16) == binding.ERR_WORKSPACE_TOO_SMALL
    # config values out of range
    cfg = binding.Config(small_cutoff=100)
    assert _call_keys(lib, aligned, 10, 4, 0, aligned, big, ctypes.byref(cfg)) == \
        binding.ERR_INVALID_ARG
    for bits in (1, 3, 9):      # a sort takes 4 .. 8 bits per pass
        cfg = binding.Config(bits_per_pass=bits)
        assert _call_keys(lib, aligned, 10, 4, 0, aligned, big, ctypes.byref(cfg)) == \
            binding.ERR_UNSUPPORTED
    # a tile other than the width's two compiled tiles (7168 / 4096 for 4-byte
    # keys alone, 4096 / 2048 and 2048 / 1024 for 8- and 16-byte keys) is refused
    for kb, wrong in ((4, 6144), (4, 3072), (4, 8192), (8, 3072), (8, 1024), (16, 4096),
                      (16, 512)):
        cfg = binding.Config(tile_keys=wrong)
        assert _call_keys(lib, aligned, 10, kb, 0, aligned, big, ctypes.byref(cfg)) == \
            binding.ERR_UNSUPPORTED
    for kb, vb in ((4, 0), (4, 4), (8, 0), (8, 8), (16, 4)):
        assert set(binding.tile_choices(kb, vb)) == \
            {7168 if (kb, vb) == (4, 0) else 6144 if kb == 4 else 4096 if kb == 8 else 2048,
             4096 if kb == 4 else 2048 if kb == 8 else 1024}
    # pairs without payload width, segmented without offsets
    assert lib.binar_sort_pairs(aligned, aligned, 10, 4, 0, 0, aligned, big, None, None) == \
        binding.ERR_INVALID_ARG
    assert lib.binar_sort_segmented(aligned, None, None, 1, 10, 4, 0, 0, aligned, big, None,
                                    None) == binding.ERR_INVALID_ARG
    # partition pass: bad bit position / digit width
    assert lib.binar_partition_pass(aligned, None, aligned, None, 10, 4, 0, 0, 32, 8, None,
                                    aligned, big, None, None) == binding.ERR_INVALID_ARG
    assert lib.binar_partition_pass(aligned, None, aligned, None, 10, 4, 0, 0, 0, 9, None,
                                    aligned, big, None, None) == binding.ERR_UNSUPPORTED
    assert lib.binar_partition_pass(aligned, None, aligned, None, 10, 4, 0, 0, 0, -1, None,
                                    aligned, big, None, None) == binding.ERR_UNSUPPORTED


def test_noalloc_debug_hook_argument_checks(lib):
    """The no-alloc pass's test hook only records its arguments (no CUDA
    call); negative values are refused and (0, 0) restores the defaults."""
    f = lib.binar_partition_pass_noalloc_debug
    f.argtypes = [ctypes.c_int, ctypes.c_int64]
    f.restype = ctypes.c_int
    assert f(-1, 0) == binding.ERR_INVALID_ARG
    assert f(0, -5) == binding.ERR_INVALID_ARG
    assert f(3, 1000) == binding.OK
    assert f(0, 0) == binding.OK


def test_wide_keys_and_strings_argument_checks(lib):
    aligned = ctypes.c_void_p(0x1000)
    big = 1 << 40
    # keys of 17 .. 256 bytes: the unsegmented sorts only, no FLOAT map
    assert _call_keys(lib, aligned, 10, 257, 3, aligned, big) == binding.ERR_INVALID_ARG
    assert _call_keys(lib, aligned, 10, 32, binding.MAP_FLOAT, aligned, big) == \
        binding.ERR_UNSUPPORTED
    assert lib.binar_sort_segmented(aligned, None, aligned, 1, 10, 32, 3, 0, aligned, big, None,
                                    None) == binding.ERR_UNSUPPORTED
    assert lib.binar_partition_pass(aligned, None, aligned, None, 10, 32, 3, 0, 0, 8, None,
                                    aligned, big, None, None) == binding.ERR_UNSUPPORTED
    assert _call_keys(lib, aligned, 1000, 64, 3, aligned, 16) == binding.ERR_WORKSPACE_TOO_SMALL
    assert binding.workspace_bytes(1000, 64, 8) > 1000 * 64
    with pytest.raises(binding.BinarError):
        binding.workspace_bytes(10, 300, 0)
    # strings: length bound, pointer alignment, workspace size
    sws = binding.strings_workspace_bytes(1000)
    assert sws > binding.strings_workspace_bytes(10) > 0
    f = lib.binar_sort_strings
    assert f(aligned, aligned, 10, binding.MAX_STRING_BYTES + 1, aligned, aligned, big, None,
             None) == binding.ERR_INVALID_ARG
    assert f(aligned, ctypes.c_void_p(0x1004), 10, 8, aligned, aligned, big, None, None) == \
        binding.ERR_INVALID_ARG
    assert f(aligned, aligned, 10, 8, ctypes.c_void_p(0x1002), aligned, big, None, None) == \
        binding.ERR_INVALID_ARG
    assert f(aligned, aligned, 1000, 8, aligned, aligned, 16, None, None) == \
        binding.ERR_WORKSPACE_TOO_SMALL


def test_inplace_argument_checks(lib):
    aligned = ctypes.c_void_p(0x1000)
    big = 1 << 40
    f = lib.binar_sort_inplace
    assert binding.inplace_workspace_bytes(1 << 20, 4, 4) < binding.workspace_bytes(1 << 20, 4, 4)
    assert f(aligned, None, 10, 32, 3, 0, aligned, big, None, None) == binding.ERR_UNSUPPORTED
    for cfg, rc in ((binding.Config(tile_keys=1024), binding.ERR_UNSUPPORTED),
                    (binding.Config(bits_per_pass=8), binding.ERR_UNSUPPORTED),
                    (binding.Config(small_cutoff=100), binding.ERR_INVALID_ARG)):
        assert f(aligned, None, 10, 4, 0, 0, aligned, big, ctypes.byref(cfg), None) == rc
    assert f(aligned, None, 100000, 4, 0, 0, aligned, 16, None, None) == \
        binding.ERR_WORKSPACE_TOO_SMALL
    assert f(aligned, aligned, 10, 4, 0, 0, aligned, big, None, None) == binding.ERR_INVALID_ARG
