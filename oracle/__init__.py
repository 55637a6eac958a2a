"""CPU oracle for binar sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
library (``paper_0811_3448_gb300``) never imports it, and it imports nothing of
the product: the two share no code.

The arithmetic lives in ``binar_oracle.c`` (plain C, built with gcc by
:func:`build`); this module only marshals numpy arrays into it.  What each
function computes, and the passage of the paper it restates:

* :func:`map_keys` -- the order-preserving encoding of a key as a big-endian bit
  string ("The Other Universal Property").
* :func:`binar_sort` -- the paper's in-place, unstable binar sort ("Operation of
  Algorithm"), per segment.  Returns the number of element placements.
* :func:`binar_sort_trace` -- the same, recording every partition configuration
  (checked against "Illustration of the Algorithm").
* :func:`binar_sort_parallel` -- the parallel variant ("Algorithm Variants"),
  for CPU timing only.
* :func:`stable_radix` -- stable binary LSD radix sort, the record-order oracle
  ("Sorting Formalism" with equal keys kept in input order).
* :func:`partition_pass` -- one stable k-bit partition at bit position ``pos``.
* :func:`sort_strings` -- the stable lexicographic order of byte strings of
  different lengths (a proper prefix first), as a permutation.
* :func:`rank_of` / :func:`occurrence` -- the output position range of one key
  and the input index of its j-th copy, by definition, for checking sampled
  outputs of sorts too large for the other functions.

Parity pins: ``tests/test_oracle_*.py`` (no GPU needed).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

MAP_UNSIGNED, MAP_SIGNED, MAP_FLOAT, MAP_BYTES_BE = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "binar_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``binar_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-Wall", "-Wextra", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def configure(lib):
    """Declares the C signatures on a loaded oracle library and returns it."""
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_map_keys.argtypes = [p, p, i64, i32, i32]
    lib.oracle_map_keys.restype = i32
    lib.oracle_binar_sort.argtypes = [p, p, p, i64, i32, i32, i32, i32]
    lib.oracle_binar_sort.restype = i64
    lib.oracle_binar_sort_trace.argtypes = [p, i64, i32, i32, i32, p, i64]
    lib.oracle_binar_sort_trace.restype = i64
    lib.oracle_binar_sort_parallel.argtypes = [p, p, i64, i32, i32, i32, i32, i32]
    lib.oracle_binar_sort_parallel.restype = i64
    lib.oracle_stable_radix.argtypes = [p, p, p, i64, i32, i32, i32, i32]
    lib.oracle_stable_radix.restype = i32
    lib.oracle_partition_pass.argtypes = [p, p, p, p, i64, i32, i32, i32, i32, i32, p]
    lib.oracle_partition_pass.restype = i32
    lib.oracle_rank_of.argtypes = [p, i64, i32, i32, p, p, p]
    lib.oracle_rank_of.restype = i32
    lib.oracle_occurrence.argtypes = [p, i64, i32, p, i64]
    lib.oracle_occurrence.restype = i64
    lib.oracle_sort_strings.argtypes = [p, p, i64, p]
    lib.oracle_sort_strings.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(build()))
    return _lib


def _key_view(keys: np.ndarray):
    """Returns (uint8 view of shape (n, kb), kb) for a C-contiguous key array.

    1-D arrays of any 1/2/4/8-byte dtype have kb = itemsize; 2-D uint8 arrays of
    shape (n, 16) are 16-byte keys."""
    if not keys.flags.c_contiguous:
        raise ValueError("keys must be C-contiguous")
    if keys.ndim == 2:
        if keys.dtype != np.uint8:
            raise ValueError("2-D keys must be uint8 of shape (n, kb)")
        return keys, keys.shape[1]
    return keys.view(np.uint8).reshape(keys.shape[0], keys.dtype.itemsize), keys.dtype.itemsize


def _vals_view(vals):
    if vals is None:
        return None, 0
    if not vals.flags.c_contiguous:
        raise ValueError("vals must be C-contiguous")
    if vals.ndim == 2:
        return vals, vals.shape[1]
    return vals.view(np.uint8).reshape(vals.shape[0], vals.dtype.itemsize), vals.dtype.itemsize


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _offsets(n, offsets):
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    if len(offsets) < 1 or offsets[0] < 0 or offsets[-1] > n or np.any(np.diff(offsets) < 0):
        raise ValueError("offsets must be nondecreasing within [0, n]")
    return offsets, len(offsets) - 1


def map_keys(keys: np.ndarray, key_map: int) -> np.ndarray:
    """Encodes keys as big-endian bit strings: returns uint8 of shape (n, kb)."""
    kv, kb = _key_view(keys)
    out = np.zeros((kv.shape[0], kb), dtype=np.uint8)
    if _load().oracle_map_keys(_ptr(kv), _ptr(out), kv.shape[0], kb, key_map) != 0:
        raise ValueError("unsupported key width / map")
    return out


def binar_sort(keys, vals=None, key_map=MAP_UNSIGNED, w=None, offsets=None):
    """Sorts ``keys`` (and ``vals`` with them) IN PLACE with the paper's binar sort.

    Returns the number of element placements (partition-loop iterations)."""
    kv, kb = _key_view(keys)
    vv, vb = _vals_view(vals)
    w = 8 * kb if w is None else w
    offs, s = _offsets(kv.shape[0], offsets)
    r = _load().oracle_binar_sort(_ptr(kv), _ptr(vv), _ptr(offs), s, kb, key_map, vb, w)
    if r < 0:
        raise ValueError("oracle_binar_sort: bad arguments")
    return int(r)


def binar_sort_trace(keys, key_map=MAP_UNSIGNED, w=None, max_rows=4096):
    """Binar sort of a small 1-byte-key array, returning every partition state.

    Each row is (pos, lower, upper, lo, hi, key bytes...)."""
    kv, kb = _key_view(keys)
    n = kv.shape[0]
    w = 8 * kb if w is None else w
    cap = max_rows * (5 + n)
    tr = np.zeros(cap, dtype=np.int64)
    used = _load().oracle_binar_sort_trace(_ptr(kv), n, kb, key_map, w, _ptr(tr), cap)
    if used < 0:
        raise ValueError("oracle_binar_sort_trace: bad arguments")
    return tr[:used].reshape(-1, 5 + n)


def binar_sort_parallel(keys, vals=None, key_map=MAP_UNSIGNED, w=None, log2_groups=4):
    """Parallel variant: split on the leading ``log2_groups`` bits, then one
    thread per group runs binar sort.  In place.  Returns placements."""
    kv, kb = _key_view(keys)
    vv, vb = _vals_view(vals)
    w = 8 * kb if w is None else w
    r = _load().oracle_binar_sort_parallel(_ptr(kv), _ptr(vv), kv.shape[0], kb, key_map,
                                           vb, w, log2_groups)
    if r < 0:
        raise ValueError("oracle_binar_sort_parallel: bad arguments")
    return int(r)


def stable_radix(keys, vals=None, key_map=MAP_UNSIGNED, w=None, offsets=None):
    """Stable binary LSD radix sort, in place, per segment."""
    kv, kb = _key_view(keys)
    vv, vb = _vals_view(vals)
    w = 8 * kb if w is None else w
    offs, s = _offsets(kv.shape[0], offsets)
    if _load().oracle_stable_radix(_ptr(kv), _ptr(vv), _ptr(offs), s, kb, key_map, vb, w) != 0:
        raise ValueError("oracle_stable_radix: bad arguments")


def partition_pass(keys, vals=None, key_map=MAP_UNSIGNED, pos=0, k=8):
    """One stable k-bit split at bit ``pos``: returns (keys_out, vals_out, offsets)."""
    kv, kb = _key_view(keys)
    vv, vb = _vals_view(vals)
    ko = np.empty_like(keys)
    kov, _ = _key_view(ko)
    vo = None if vals is None else np.empty_like(vals)
    vov, _ = _vals_view(vo)
    offs = np.zeros((1 << k) + 1, dtype=np.int64)
    if _load().oracle_partition_pass(_ptr(kv), _ptr(vv), _ptr(kov), _ptr(vov), kv.shape[0], kb,
                                     key_map, vb, pos, k, _ptr(offs)) != 0:
        raise ValueError("oracle_partition_pass: bad arguments")
    return ko, vo, offs


def rank_of(keys, probe, key_map=MAP_UNSIGNED):
    """(number of keys below probe, number not above probe) by the encoding."""
    kv, kb = _key_view(keys)
    pr = np.ascontiguousarray(np.asarray(probe)).view(np.uint8).reshape(-1)
    if pr.shape[0] != kb:
        raise ValueError("probe must be one key")
    lt, le = ctypes.c_int64(0), ctypes.c_int64(0)
    if _load().oracle_rank_of(_ptr(kv), kv.shape[0], kb, key_map, _ptr(pr), ctypes.byref(lt),
                              ctypes.byref(le)) != 0:
        raise ValueError("oracle_rank_of: bad arguments")
    return lt.value, le.value


def occurrence(keys, probe, j):
    """Input index of the j-th (0-based) key bit-identical to probe, or -1."""
    kv, kb = _key_view(keys)
    pr = np.ascontiguousarray(np.asarray(probe)).view(np.uint8).reshape(-1)
    return int(_load().oracle_occurrence(_ptr(kv), kv.shape[0], kb, _ptr(pr), j))


def sort_strings(data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Stable lexicographic order of the strings data[offsets[i]:offsets[i+1]]
    (unsigned bytes, a proper prefix first): returns uint32 indices."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    if n < 0 or (n > 0 and (offsets[0] < 0 or offsets[-1] > len(data))):
        raise ValueError("offsets must lie within the byte buffer")
    order = np.zeros(max(n, 0), dtype=np.uint32)
    if _load().oracle_sort_strings(_ptr(data), _ptr(offsets), n, _ptr(order)) != 0:
        raise ValueError("oracle_sort_strings: bad arguments")
    return order
