"""Helpers shared by the GPU parity tests (torch <-> numpy, oracle calls)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

MAPS = {np.dtype(np.uint32): oracle.MAP_UNSIGNED, np.dtype(np.uint64): oracle.MAP_UNSIGNED,
        np.dtype(np.int32): oracle.MAP_SIGNED, np.dtype(np.int64): oracle.MAP_SIGNED,
        np.dtype(np.float32): oracle.MAP_FLOAT, np.dtype(np.float64): oracle.MAP_FLOAT}


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def key_map_of(keys: np.ndarray) -> int:
    if keys.ndim == 2:
        return oracle.MAP_BYTES_BE
    return MAPS[keys.dtype]


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy()


def expect_keys(keys: np.ndarray) -> np.ndarray:
    k = keys.copy()
    oracle.binar_sort(k, key_map=key_map_of(keys))
    return k


def expect_pairs(keys: np.ndarray, vals: np.ndarray, offsets=None):
    k, v = keys.copy(), vals.copy()
    oracle.stable_radix(k, v, key_map=key_map_of(keys), offsets=offsets)
    return k, v


def same_bits(a: np.ndarray, b: np.ndarray) -> bool:
    return a.shape == b.shape and np.array_equal(np.ascontiguousarray(a).view(np.uint8),
                                                 np.ascontiguousarray(b).view(np.uint8))
