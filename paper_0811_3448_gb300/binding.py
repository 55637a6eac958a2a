"""ctypes binding of libbinar (include/binar.h) for torch tensors.

Argument marshalling only: every step of a sort runs in the CUDA kernels of
``libbinar.so``.  torch provides device memory (tensors, the workspace) and the
stream (``torch.cuda.current_stream()``).  If the library is missing this module
raises; there is no other implementation to fall back to.

Key types and their default key-to-bits map (binar_key_map):

=================  ==========  ==============
tensor             key_bytes   default map
=================  ==========  ==============
uint32 / uint64    4 / 8       UNSIGNED
int32 / int64      4 / 8       SIGNED
float32 / float64  4 / 8       FLOAT
uint8 of (n, 16)   16          BYTES_BE
uint8 of (n, kb)   17 .. 256   BYTES_BE (sort_keys / sort_pairs only)
=================  ==========  ==============

Byte strings of different lengths: :func:`sort_strings` (bytes + offsets,
returns the order).

Payloads: any 4- or 8-byte dtype (moved as opaque bits).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

MAP_UNSIGNED, MAP_SIGNED, MAP_FLOAT, MAP_BYTES_BE = 0, 1, 2, 3
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE_TOO_SMALL = 0, 1, 2, 3
ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_DEVICE_BOUNDS, ERR_QUEUE_OVERFLOW = 4, 5, 6, 7
MAX_BUCKET_KEYS = 2147483646
MAX_KEY_BYTES = 256
MAX_STRING_BYTES = 4096

_lib = None
_lock = threading.Lock()


class BinarError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = load().binar_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


class Config(ctypes.Structure):
    """binar_config: zero fields take the library defaults."""
    _fields_ = [("tile_keys", ctypes.c_int), ("bits_per_pass", ctypes.c_int),
                ("small_cutoff", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("lookback_timeout_ns", ctypes.c_int64),
                ("debug_skip_publish_tile", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def load():
    """Opens libbinar.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libbinar not built: {path} is missing")
        lib = ctypes.CDLL(path)
        p, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        cfgp = ctypes.POINTER(Config)
        lib.binar_workspace_bytes.argtypes = [i64, i64, i32, i32, ctypes.POINTER(sz)]
        lib.binar_sort_keys.argtypes = [p, i64, i32, i32, p, sz, cfgp, p]
        lib.binar_sort_pairs.argtypes = [p, p, i64, i32, i32, i32, p, sz, cfgp, p]
        lib.binar_sort_segmented.argtypes = [p, p, p, i64, i64, i32, i32, i32, p, sz, cfgp, p]
        lib.binar_partition_pass.argtypes = [p, p, p, p, i64, i32, i32, i32, i32, i32, p, p, sz,
                                             cfgp, p]
        lib.binar_workspace_status.argtypes = [p, p, ctypes.POINTER(i32)]
        lib.binar_status_string.argtypes = [i32]
        lib.binar_status_string.restype = ctypes.c_char_p
        lib.binar_profile_start.argtypes = []
        lib.binar_profile_stop.argtypes = [ctypes.POINTER(KernelStat), i32, ctypes.POINTER(i32)]
        lib.binar_version.restype = ctypes.c_char_p
        lib.binar_generate.argtypes = [p, i64, i32, ctypes.c_uint64, p]
        lib.binar_strings_workspace_bytes.argtypes = [i64, ctypes.POINTER(sz)]
        lib.binar_inplace_workspace_bytes.argtypes = [i64, i32, i32, cfgp, ctypes.POINTER(sz)]
        lib.binar_sort_inplace.argtypes = [p, p, i64, i32, i32, i32, p, sz, cfgp, p]
        lib.binar_sort_strings.argtypes = [p, p, i64, i64, p, p, sz, cfgp, p]
        for name in ("binar_workspace_bytes", "binar_sort_keys", "binar_sort_pairs",
                     "binar_sort_segmented", "binar_partition_pass", "binar_workspace_status",
                     "binar_profile_start", "binar_profile_stop", "binar_generate",
                     "binar_strings_workspace_bytes", "binar_sort_strings",
                     "binar_inplace_workspace_bytes", "binar_sort_inplace"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


# Keys per partition tile of the two compiled tile shapes (binar_config.tile_keys):
# by key width, and for 4-byte keys by whether a payload moves with them.
_TILES = {(4, False): (7168, 4096), (4, True): (6144, 4096), (8, False): (4096, 2048),
          (8, True): (4096, 2048), (16, False): (2048, 1024), (16, True): (2048, 1024)}
MIN_SORT_BITS, MAX_BITS = 4, 8


def tile_choices(key_bytes: int, val_bytes: int = 0):
    """The tile sizes binar_config.tile_keys accepts for this shape (default first)."""
    return _TILES[(key_bytes, val_bytes > 0)]


# ------------------------------------------------------------------ helpers
_DEFAULT_MAP = {torch.uint32: MAP_UNSIGNED, torch.uint64: MAP_UNSIGNED,
                torch.int32: MAP_SIGNED, torch.int64: MAP_SIGNED,
                torch.float32: MAP_FLOAT, torch.float64: MAP_FLOAT}


def key_layout(keys: torch.Tensor):
    """(n, key_bytes, default map) of a key tensor."""
    if keys.dim() == 2 and keys.dtype == torch.uint8 and 16 <= keys.shape[1] <= MAX_KEY_BYTES:
        return keys.shape[0], keys.shape[1], MAP_BYTES_BE
    if keys.dim() != 1 or keys.dtype not in _DEFAULT_MAP:
        raise TypeError(f"unsupported key tensor {keys.dtype} {tuple(keys.shape)}")
    return keys.shape[0], keys.element_size(), _DEFAULT_MAP[keys.dtype]


def _val_bytes(vals):
    if vals is None:
        return 0
    if vals.dim() != 1 or vals.element_size() not in (4, 8):
        raise TypeError("payloads must be a 1-D tensor of a 4- or 8-byte dtype")
    return vals.element_size()


def _check_dev(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("tensors must be contiguous CUDA tensors")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _cfg(config):
    if config is None:
        return None
    if isinstance(config, Config):
        return ctypes.byref(config)
    return ctypes.byref(Config(**config))


def _check(rc, what):
    if rc != OK:
        raise BinarError(rc, what)


def workspace_bytes(n: int, key_bytes: int, val_bytes: int = 0, num_segments: int = 1) -> int:
    out = ctypes.c_size_t(0)
    _check(load().binar_workspace_bytes(n, num_segments, key_bytes, val_bytes, ctypes.byref(out)),
           "binar_workspace_bytes")
    return out.value


def workspace(n: int, key_bytes: int, val_bytes: int = 0, num_segments: int = 1,
              device=None) -> torch.Tensor:
    """A workspace tensor large enough for one call of that shape."""
    nbytes = workspace_bytes(n, key_bytes, val_bytes, num_segments)
    return torch.empty(max(nbytes, 16), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def _ws_for(ws, n, kb, vb, segs, device):
    if ws is None:
        ws = workspace(n, kb, vb, segs, device)
    _check_dev(ws)
    return ws


# ------------------------------------------------------------------ calls
def sort_keys(keys: torch.Tensor, key_map=None, ws=None, config=None, stream=None) -> torch.Tensor:
    """Sorts ``keys`` in place (binar_sort_keys) and returns it."""
    _check_dev(keys)
    n, kb, dmap = key_layout(keys)
    ws = _ws_for(ws, n, kb, 0, 1, keys.device)
    _check(load().binar_sort_keys(_ptr(keys), n, kb, dmap if key_map is None else key_map,
                                  _ptr(ws), ws.numel(), _cfg(config), _stream(stream)),
           "binar_sort_keys")
    return keys


def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_map=None, ws=None, config=None,
               stream=None):
    """Sorts records (keys, vals) in place, stably (binar_sort_pairs)."""
    _check_dev(keys, vals)
    n, kb, dmap = key_layout(keys)
    vb = _val_bytes(vals)
    if vals.shape[0] != n:
        raise ValueError("keys and vals differ in length")
    ws = _ws_for(ws, n, kb, vb, 1, keys.device)
    _check(load().binar_sort_pairs(_ptr(keys), _ptr(vals), n, kb,
                                   dmap if key_map is None else key_map, vb, _ptr(ws),
                                   ws.numel(), _cfg(config), _stream(stream)),
           "binar_sort_pairs")
    return keys, vals


def sort_segmented(keys: torch.Tensor, offsets: torch.Tensor, vals: torch.Tensor = None,
                   key_map=None, ws=None, config=None, stream=None):
    """Sorts every segment [offsets[s], offsets[s+1]) in place (binar_sort_segmented)."""
    _check_dev(keys, vals, offsets)
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or offsets.shape[0] < 1:
        raise TypeError("offsets must be a 1-D int64 CUDA tensor of num_segments+1 entries")
    n, kb, dmap = key_layout(keys)
    vb = _val_bytes(vals)
    segs = offsets.shape[0] - 1
    ws = _ws_for(ws, n, kb, vb, max(segs, 1), keys.device)
    _check(load().binar_sort_segmented(_ptr(keys), _ptr(vals), _ptr(offsets), segs, n, kb,
                                       dmap if key_map is None else key_map, vb, _ptr(ws),
                                       ws.numel(), _cfg(config), _stream(stream)),
           "binar_sort_segmented")
    return keys, vals


def partition_pass(keys: torch.Tensor, vals: torch.Tensor = None, pos: int = 0, key_map=None,
                   ws=None, config=None, stream=None, out=None, bits: int = 8):
    """One stable partition pass on the ``bits`` (1 .. 8) key bits at bit
    ``pos``, out of place.  Returns (keys_out, vals_out, offsets[2^bits + 1])."""
    _check_dev(keys, vals)
    n, kb, dmap = key_layout(keys)
    vb = _val_bytes(vals)
    if out is None:
        ko = torch.empty_like(keys)
        vo = None if vals is None else torch.empty_like(vals)
        offs = torch.empty((1 << bits) + 1, dtype=torch.int64, device=keys.device)
    else:
        ko, vo, offs = out
    ws = _ws_for(ws, n, kb, vb, 1, keys.device)
    _check(load().binar_partition_pass(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, kb,
                                       dmap if key_map is None else key_map, vb, pos, bits,
                                       _ptr(offs), _ptr(ws), ws.numel(), _cfg(config),
                                       _stream(stream)),
           "binar_partition_pass")
    return ko, vo, offs


def inplace_workspace_bytes(n: int, key_bytes: int, val_bytes: int = 0, config=None) -> int:
    out = ctypes.c_size_t(0)
    _check(load().binar_inplace_workspace_bytes(n, key_bytes, val_bytes, _cfg(config),
                                                ctypes.byref(out)),
           "binar_inplace_workspace_bytes")
    return out.value


def sort_inplace(keys: torch.Tensor, vals: torch.Tensor = None, key_map=None, ws=None,
                 config=None, stream=None):
    """Sorts keys (and payloads) in place and unstably (binar_sort_inplace):
    the paper's one-bit exchange passes, no second array."""
    _check_dev(keys, vals)
    n, kb, dmap = key_layout(keys)
    vb = _val_bytes(vals)
    if vals is not None and vals.shape[0] != n:
        raise ValueError("keys and vals differ in length")
    if ws is None:
        ws = torch.empty(max(inplace_workspace_bytes(n, kb, vb, config), 16), dtype=torch.uint8,
                         device=keys.device)
    _check_dev(ws)
    _check(load().binar_sort_inplace(_ptr(keys), _ptr(vals), n, kb,
                                     dmap if key_map is None else key_map, vb, _ptr(ws),
                                     ws.numel(), _cfg(config), _stream(stream)),
           "binar_sort_inplace")
    return keys, vals


def strings_workspace_bytes(n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().binar_strings_workspace_bytes(n, ctypes.byref(out)),
           "binar_strings_workspace_bytes")
    return out.value


def sort_strings(data: torch.Tensor, offsets: torch.Tensor, max_len: int = None, ws=None,
                 config=None, stream=None, order=None) -> torch.Tensor:
    """Stable lexicographic order of the byte strings data[offsets[i]:offsets[i+1]]
    (binar_sort_strings): returns int32 indices (read as uint32) of the strings
    in order.  ``max_len`` bounds every string's length (default: computed
    from ``offsets``, which synchronises)."""
    _check_dev(data, offsets)
    if data.dtype != torch.uint8 or data.dim() != 1:
        raise TypeError("data must be a 1-D uint8 CUDA tensor")
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or offsets.shape[0] < 1:
        raise TypeError("offsets must be a 1-D int64 CUDA tensor of n + 1 entries")
    n = offsets.shape[0] - 1
    if max_len is None:
        max_len = int((offsets[1:] - offsets[:-1]).max().item()) if n > 0 else 0
    if order is None:
        order = torch.empty(n, dtype=torch.int32, device=data.device)
    if ws is None:
        ws = torch.empty(max(strings_workspace_bytes(n), 16), dtype=torch.uint8,
                         device=data.device)
    _check_dev(ws, order)
    _check(load().binar_sort_strings(_ptr(data), _ptr(offsets), n, max_len, _ptr(order),
                                     _ptr(ws), ws.numel(), _cfg(config), _stream(stream)),
           "binar_sort_strings")
    return order


def workspace_status(ws: torch.Tensor, stream=None) -> int:
    """Synchronises the stream and returns (and clears) the device status word."""
    st = ctypes.c_int(0)
    _check(load().binar_workspace_status(_ptr(ws), _stream(stream), ctypes.byref(st)),
           "binar_workspace_status")
    return st.value


def check_status(ws: torch.Tensor, stream=None) -> None:
    st = workspace_status(ws, stream)
    if st != OK:
        raise BinarError(st, "device")


def status_string(status: int) -> str:
    return load().binar_status_string(status).decode()


def profile_start() -> None:
    _check(load().binar_profile_start(), "binar_profile_start")


def profile_stop():
    """Returns {kernel name: (launches, total_ms)} since profile_start()."""
    cap = 256
    arr = (KernelStat * cap)()
    cnt = ctypes.c_int(0)
    _check(load().binar_profile_stop(arr, cap, ctypes.byref(cnt)), "binar_profile_stop")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(cnt.value, cap))}


def generate(out: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Fills ``out`` (4-, 8- or 16-byte elements; uint8 (n, 16) for 16) with
    SplitMix64 values of counters 0 .. n-1 (binar_generate)."""
    _check_dev(out)
    if out.dim() == 2 and out.dtype == torch.uint8 and out.shape[1] == 16:
        n, eb = out.shape[0], 16
    elif out.dim() == 1 and out.element_size() in (4, 8):
        n, eb = out.shape[0], out.element_size()
    else:
        raise TypeError("generate: 1-D 4/8-byte tensor or uint8 (n, 16)")
    _check(load().binar_generate(_ptr(out), n, eb, ctypes.c_uint64(seed & (2**64 - 1)),
                                 _stream(stream)), "binar_generate")
    return out


def version() -> str:
    return load().binar_version().decode()
