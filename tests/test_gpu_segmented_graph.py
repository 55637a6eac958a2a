"""Segmented sort (config 4 recipe) captured in a CUDA graph.

The whole segmented sort -- every kernel of every level -- is enqueued by one
binar_sort_segmented call with no host synchronisation, so it can be captured
once and replayed.  Checks: the replayed graph gives the same bytes as direct
calls and as one binar_sort_pairs call per segment, and the output is the
stable per-segment sort (properties that fix it at any size)."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _segment_case(total, count, seed_variant=0):
    sizes = inputs.config4_segment_sizes(total=total, count=count, variant=seed_variant)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(4 + seed_variant)))
    keys[::7] = keys[3]           # duplicates across and inside segments
    vals = inputs.segment_index_payload(off)
    return off, keys, vals


def _check_segments(torch, off_np, k_in, k_out, v_out):
    n = k_out.shape[0]
    off = torch.from_numpy(off_np).cuda()
    seg = torch.repeat_interleave(torch.arange(len(off_np) - 1, device="cuda"),
                                  off[1:] - off[:-1])
    k = k_out.to(torch.int64)
    v = v_out.to(torch.int64)
    same = seg[1:] == seg[:-1]
    assert bool((k[1:][same] >= k[:-1][same]).all()), "segment not sorted"
    gidx = off[:-1][seg] + v
    assert bool((torch.bincount(gidx, minlength=n) == 1).all()), "payload not a permutation"
    assert bool((k_in.to(torch.int64)[gidx] == k).all()), "key / payload mismatch"
    eq = same & (k[1:] == k[:-1])
    assert bool((v[1:][eq] > v[:-1][eq]).all()), "equal keys out of input order"


def test_graph_replay_equals_direct_and_per_segment_calls():
    require_gpu()
    torch = pytest.importorskip("torch")
    off, keys, vals = _segment_case(total=8 << 20, count=2000)
    n = int(off[-1])
    toff = to_dev(off)
    ws = binding.workspace(n, 4, 4, len(off) - 1)
    # direct call
    dk, dv = to_dev(keys), to_dev(vals)
    binding.sort_segmented(dk, toff, dv, ws=ws)
    binding.check_status(ws)
    # one call per segment (the plain form)
    pk, pv = to_dev(keys), to_dev(vals)
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        if b - a >= 2:
            binding.sort_pairs(pk[a:b], pv[a:b], ws=ws)
    binding.check_status(ws)
    # captured graph, replayed twice over fresh inputs
    gk, gv = to_dev(keys), to_dev(vals)
    src_k, src_v = to_dev(keys), to_dev(vals)
    binding.sort_segmented(gk, toff, gv, ws=ws)     # first call on the device: set-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            binding.sort_segmented(gk, toff, gv, ws=ws)
    for _ in range(2):
        gk.copy_(src_k)
        gv.copy_(src_v)
        graph.replay()
        torch.cuda.synchronize()
        assert same_bits(to_host(gk), to_host(dk)) and same_bits(to_host(gv), to_host(dv))
    assert binding.workspace_status(ws) == binding.OK
    assert same_bits(to_host(pk), to_host(dk)) and same_bits(to_host(pv), to_host(dv))
    # and the oracle on a sample of segments
    for s in range(0, len(off) - 1, 97):
        a, b = int(off[s]), int(off[s + 1])
        ek, ev = keys[a:b].copy(), vals[a:b].copy()
        oracle.stable_radix(ek, ev)
        assert same_bits(to_host(dk[a:b]), ek) and same_bits(to_host(dv[a:b]), ev)


def test_config4_full_size_graph():
    """20,000 log-uniform segments, about 256M uint32 keys, one graph launch."""
    require_gpu()
    torch = pytest.importorskip("torch")
    off, keys, vals = _segment_case(total=256 << 20, count=20000, seed_variant=1)
    n = int(off[-1])
    toff = to_dev(off)
    k_in = to_dev(keys)
    gk, gv = k_in.clone(), to_dev(vals)
    src_v = gv.clone()
    ws = binding.workspace(n, 4, 4, len(off) - 1)
    binding.sort_segmented(gk, toff, gv, ws=ws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            binding.sort_segmented(gk, toff, gv, ws=ws)
    gk.copy_(k_in)
    gv.copy_(src_v)
    graph.replay()
    torch.cuda.synchronize()
    assert binding.workspace_status(ws) == binding.OK
    _check_segments(torch, off, k_in, gk, gv)
