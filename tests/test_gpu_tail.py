"""The fused level tail of small sorts: for sorts of at most 2^21 keys with
the default tile, the levels after the first run as one cooperative launch
(grid barriers between the phases) that ends at the first level without a
bucket.  Checked against the oracle on inputs whose tail has no work
(uniform) and real work at several levels (shared prefixes, few bits per
pass, a small cutoff, heavy duplicates); that the call makes one tail launch
and no per-level launches after level 0, while 2^21 + 1 keys or the second
tile shape keep the per-level launches; and that a captured CUDA graph with
a working tail replays correctly."""
import numpy as np
import pytest

from gpu_util import expect_keys, expect_pairs, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LIMIT = 1 << 21


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _launches(fn):
    binding.profile_start()
    fn()
    torch.cuda.synchronize()
    return binding.profile_stop()


def _sort_pairs(keys, vals, config=None):
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(len(keys), keys.itemsize, vals.itemsize)
    stats = _launches(lambda: binding.sort_pairs(tk, tv, ws=ws, config=config))
    binding.check_status(ws)
    return to_host(tk), to_host(tv), stats


def _prefixed(n, bits, seed, dtype=np.uint32):
    """Keys whose top `bits` bits take only a few values: buckets stay large
    for several levels."""
    g = np.random.Generator(np.random.PCG64(seed))
    w = np.dtype(dtype).itemsize * 8
    low = inputs.uniform_keys(n, dtype, g) >> dtype(bits)
    top = g.integers(0, 3, size=n).astype(dtype) << dtype(w - bits)
    return (top | low).astype(dtype)


@pytest.mark.parametrize("n", [70_001, 1 << 20, LIMIT])
def test_uniform_tail_is_one_launch(n):
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(n)))
    vals = inputs.index_payload(n)
    k, v, stats = _sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert stats.get("levels[1]", (0,))[0] == 1, stats
    per_level = ("prep[", "hist[", "classify[", "partition[")
    assert not any(name.startswith(per_level) and not name.endswith("[0]") for name in stats), stats


@pytest.mark.parametrize("case", ["prefix12_k8", "prefix20_k6", "cutoff2048_k4", "zipf", "u64_prefix"])
def test_tail_with_work(case):
    n = 900_001
    cfg = None
    if case == "prefix12_k8":
        keys = _prefixed(n, 12, 1)
    elif case == "prefix20_k6":
        keys, cfg = _prefixed(n, 20, 2), {"bits_per_pass": 6}
    elif case == "cutoff2048_k4":
        keys, cfg = _prefixed(n, 8, 3), {"bits_per_pass": 4, "small_cutoff": 2048}
    elif case == "zipf":
        keys = inputs.config2_keys(n, np.uint32, "zipf")
    else:
        keys = _prefixed(n, 40, 4, np.uint64)
    vals = inputs.index_payload(n)
    k, v, stats = _sort_pairs(keys, vals, cfg)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert "levels[1]" in stats, stats
    t = to_dev(keys)
    ws = binding.workspace(n, keys.itemsize, 0)
    binding.sort_keys(t, ws=ws, config=cfg)
    binding.check_status(ws)
    assert same_bits(to_host(t), expect_keys(keys))


def test_per_level_launches_above_the_bound_and_for_the_second_tile():
    n = LIMIT + 1
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(9)))
    vals = inputs.index_payload(n)
    k, v, stats = _sort_pairs(keys, vals)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert "levels[1]" not in stats and "partition[1]" in stats
    m = 500_001
    keys = _prefixed(m, 12, 5)
    vals = inputs.index_payload(m)
    k, v, stats = _sort_pairs(keys, vals, {"tile_keys": binding.tile_choices(4, 4)[1]})
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(k, ek) and same_bits(v, ev)
    assert "levels[1]" not in stats and "partition[1]" in stats


def test_graph_replay_with_a_working_tail():
    n = 1 << 20
    keys = _prefixed(n, 16, 6)
    vals = inputs.index_payload(n)
    k0, v0 = to_dev(keys), to_dev(vals)
    k, v = torch.empty_like(k0), torch.empty_like(v0)
    ws = binding.workspace(n, 4, 4)
    ek, ev = expect_pairs(keys, vals)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        k.copy_(k0)
        v.copy_(v0)
        binding.sort_pairs(k, v, ws=ws)             # set-up before capture
        with torch.cuda.graph(graph, stream=s):
            binding.sort_pairs(k, v, ws=ws)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        k.copy_(k0)
        v.copy_(v0)
        graph.replay()
    torch.cuda.synchronize()
    binding.check_status(ws)
    assert same_bits(to_host(k), ek) and same_bits(to_host(v), ev)
