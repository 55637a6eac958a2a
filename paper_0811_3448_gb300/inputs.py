"""Seeded synthetic inputs for binar sort.

This module holds no sorting arithmetic: it only draws keys, payloads,
segment sizes and request mixes from seeded generators, so that the tests can
feed the same arrays to the CUDA library and to the CPU oracle.  It imports
numpy only.

Seeds: base 8113448; seed = base + 100 * config + variant (one numpy PCG64
stream per array).  Workloads (sizes are parameters so that tests can draw the
same recipe at small n):

* config 1 -- uniform uint32 keys over [0, 2^32).
* config 2 -- uint32 / uint64 keys with a uint32 payload equal to the original
  index; distributions "uniform", "zipf" (s = 1.2 over 2^20 distinct values of
  the key width), "distinct8" (8 values drawn from the key domain, each key one
  of them uniformly), "sorted" (ascending uniform), "reverse" (descending).
* config 3 -- float32 mixture (96 % N(0,1); 0.5 % each of +0, -0, +inf, -inf;
  1 % denormals with a random non-zero mantissa and sign; 1 % exact duplicates
  of other elements; positions shuffled), uniform signed int64, uniform 16-byte
  strings, and 16-byte strings sharing one random 12-byte prefix.
* config 4 -- 20 000 segment sizes floor(2^(20 U)) rescaled so that they sum to
  about the requested total (each at least 1), in draw order.
* config 5 -- serving requests: Poisson arrivals, sizes floor(2^(10 + 16 U)),
  key type uniform over {uint32, uint64, float32}, payload with probability 1/2.

Device-side request data (config 5) comes from a counter-based generator,
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): value(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)
with mix(z) = z ^ z>>31 after z = (z ^ z>>30) * 0xBF58476D1CE4E5B9 and
z = (z ^ z>>27) * 0x94D049BB133111EB.  :func:`splitmix64` is the host
restatement used to check requests generated on the device.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 8113448
KEY_DTYPES = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32,
              "i32": np.int32, "f64": np.float64}


def seed_of(config: int, variant: int = 0) -> int:
    return BASE_SEED + 100 * config + variant


def rng(config: int, variant: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_of(config, variant)))


def uniform_keys(n: int, dtype, g: np.random.Generator) -> np.ndarray:
    """n keys uniform over every bit pattern of the dtype (integers) or, for
    floats, over every finite-or-not bit pattern."""
    dt = np.dtype(dtype)
    return np.frombuffer(g.bytes(n * dt.itemsize), dtype=dt).copy()


def config1_keys(n: int = 1 << 20) -> np.ndarray:
    """Config 1: uniform uint32 keys."""
    return uniform_keys(n, np.uint32, rng(1))


_DIST_VARIANT = {"uniform": 0, "zipf": 1, "distinct8": 2, "sorted": 3, "reverse": 4}


def _distinct_values(count: int, dtype, g: np.random.Generator) -> np.ndarray:
    out = np.empty(0, dtype=dtype)
    while out.shape[0] < count:
        more = uniform_keys(2 * count, dtype, g)
        cat = np.concatenate([out, more])
        _, first = np.unique(cat, return_index=True)
        out = cat[np.sort(first)]
    return out[:count]


def zipf_ranks(n: int, g: np.random.Generator, s: float = 1.2, support: int = 1 << 20) -> np.ndarray:
    """Ranks in [0, support) with P(r) proportional to (r + 1)^-s."""
    p = np.arange(1, support + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    u = g.random(n)
    return np.minimum(np.searchsorted(cdf, u, side="right"), support - 1)


def config2_keys(n: int, dtype=np.uint32, dist: str = "uniform") -> np.ndarray:
    """Config 2 keys (payload is np.arange(n, dtype=uint32))."""
    variant = _DIST_VARIANT[dist] + (10 if np.dtype(dtype).itemsize == 8 else 0)
    g = rng(2, variant)
    if dist == "uniform":
        return uniform_keys(n, dtype, g)
    if dist == "zipf":
        values = _distinct_values(1 << 20, dtype, g)
        return values[zipf_ranks(n, g)]
    if dist == "distinct8":
        values = _distinct_values(8, dtype, g)
        return values[g.integers(0, 8, size=n)]
    if dist == "sorted":
        return np.sort(uniform_keys(n, dtype, g))
    if dist == "reverse":
        return np.sort(uniform_keys(n, dtype, g))[::-1].copy()
    raise ValueError(dist)


def index_payload(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def config3_f32(n: int) -> np.ndarray:
    """Config 3 float32 mixture (bit patterns of the specials are exact)."""
    g = rng(3, 0)
    x = g.standard_normal(n).astype(np.float32)
    bits = x.view(np.uint32)
    kind = g.random(n)
    # 0.5 % each: +0, -0, +inf, -inf; 1 % denormals; 1 % duplicates
    edges = np.cumsum([0.005, 0.005, 0.005, 0.005, 0.01, 0.01])
    bits[kind < edges[0]] = 0x00000000
    bits[(kind >= edges[0]) & (kind < edges[1])] = 0x80000000
    bits[(kind >= edges[1]) & (kind < edges[2])] = 0x7F800000
    bits[(kind >= edges[2]) & (kind < edges[3])] = 0xFF800000
    den = (kind >= edges[3]) & (kind < edges[4])
    nd = int(den.sum())
    mant = g.integers(1, 1 << 23, size=nd, dtype=np.uint32)
    sign = g.integers(0, 2, size=nd, dtype=np.uint32) << np.uint32(31)
    bits[den] = mant | sign
    dup = (kind >= edges[4]) & (kind < edges[5])
    nz = int(dup.sum())
    if nz and n > 1:
        src = g.integers(0, n, size=nz)
        bits[dup] = bits[src]
    perm = g.permutation(n)
    return bits[perm].view(np.float32).copy()


def config3_i64(n: int) -> np.ndarray:
    return uniform_keys(n, np.int64, rng(3, 1))


def config3_bytes16(n: int, shared_prefix: bool = False) -> np.ndarray:
    """16-byte keys as uint8 of shape (n, 16); optionally one shared 12-byte prefix."""
    g = rng(3, 3 if shared_prefix else 2)
    k = g.integers(0, 256, size=(n, 16), dtype=np.uint8)
    if shared_prefix:
        k[:, :12] = g.integers(0, 256, size=12, dtype=np.uint8)
    return k


def config4_segment_sizes(total: int = 256 << 20, count: int = 20000, max_log2: int = 20,
                          variant: int = 0) -> np.ndarray:
    """Segment sizes floor(2^(max_log2 * U)) rescaled to sum to about `total`."""
    g = rng(4, variant)
    raw = np.floor(2.0 ** (max_log2 * g.random(count)))
    scaled = np.floor(raw * (total / raw.sum())).astype(np.int64)
    return np.maximum(scaled, 1)


def wide_keys(n: int, key_bytes: int, shared_prefix: int = 0, variant: int = 0) -> np.ndarray:
    """Fixed-width byte-string keys longer than 16 bytes, uint8 of shape
    (n, key_bytes), uniform bytes; optionally the first `shared_prefix` bytes
    are one random prefix shared by every key."""
    g = rng(6, variant)
    k = g.integers(0, 256, size=(n, key_bytes), dtype=np.uint8)
    if shared_prefix:
        k[:, :shared_prefix] = g.integers(0, 256, size=shared_prefix, dtype=np.uint8)
    return k


def strings(n: int, max_len: int = 64, min_len: int = 0, alphabet: int = 256,
            shared_prefix: int = 0, variant: int = 0):
    """Variable-length byte strings: lengths uniform in [min_len, max_len],
    bytes uniform over the first `alphabet` byte values; optionally every
    string starts with (the first bytes of) one random prefix of
    `shared_prefix` bytes.  Returns (bytes uint8, offsets int64 of n + 1)."""
    g = rng(7, variant)
    lens = g.integers(min_len, max_len + 1, size=n).astype(np.int64)
    off = offsets_from_sizes(lens)
    data = g.integers(0, alphabet, size=int(off[-1]), dtype=np.uint8)
    if shared_prefix:
        pre = g.integers(0, alphabet, size=shared_prefix, dtype=np.uint8)
        take = np.minimum(lens, shared_prefix)
        idx = np.repeat(off[:-1], take) + (np.arange(int(take.sum())) -
                                          np.repeat(np.cumsum(take) - take, take))
        data[idx] = pre[idx - np.repeat(off[:-1], take)]
    return data, off


def offsets_from_sizes(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def segment_index_payload(offsets: np.ndarray) -> np.ndarray:
    """Payload = index of the element within its segment."""
    n = int(offsets[-1])
    seg_start = np.repeat(offsets[:-1], np.diff(offsets))
    return (np.arange(n, dtype=np.int64) - seg_start).astype(np.uint32)


SERVE_KEY_TYPES = ("u32", "u64", "f32")


def config5_requests(rate_hz: float = 2000.0, duration_s: float = 60.0, min_log2: int = 10,
                     span_log2: int = 16, variant: int = 0):
    """Request mix: list of dicts (arrival_s, n, key_type, has_payload, seed)."""
    g = rng(5, variant)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(np.floor(2.0 ** (min_log2 + span_log2 * g.random())))
        kt = SERVE_KEY_TYPES[int(g.integers(0, 3))]
        out.append({"arrival_s": t, "n": n, "key_type": kt,
                    "has_payload": bool(g.random() < 0.5),
                    "seed": int(g.integers(0, 2**62))})
    return out


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """SplitMix64 outputs for counters start .. start+n-1 (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))
