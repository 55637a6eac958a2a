"""Serving loop on the GPU: device-generated inputs match the host definition,
every request's result is the same alone and inside a mixed batch (tolerance
0: bit-identical), sampled results equal the oracle, and a request above the
budget is rejected while the rest are served."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, same_bits, to_host
from paper_0811_3448_gb300 import binding, inputs, serve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eb", [4, 8, 16])
@pytest.mark.parametrize("n", [1, 1000, 300_001])
def test_generate_matches_host_splitmix64(eb, n):
    require_gpu()
    torch = pytest.importorskip("torch")
    seed = 0x1234_5678_9ABC_DEF0
    if eb == 16:
        out = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    else:
        out = torch.empty(n, dtype=torch.uint32 if eb == 4 else torch.uint64, device="cuda")
    binding.generate(out, seed)
    got = to_host(out)
    x = inputs.splitmix64(seed, n)
    if eb == 4:
        want = (x & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    elif eb == 8:
        want = x
    else:
        y = inputs.splitmix64(seed ^ 0xD1B54A32D192ED03, n)
        want = np.stack([x, y], axis=1).astype("<u8").view(np.uint8).reshape(n, 16)
    assert same_bits(got, want)


def _mix(count=60, seed=11):
    g = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(count):
        n = int(2 ** (10 + 11 * g.random()))            # 1K .. 2M keys
        reqs.append(serve.Request(rid=i, n=n, key_type=("u32", "u64", "f32")[i % 3],
                                  has_payload=bool(g.random() < 0.5),
                                  seed=int(g.integers(0, 2**62)),
                                  arrival_s=0.002 * (i // 10)))   # bursts of 10
    return reqs


def _host_reference(r):
    """The request's input regenerated on the host and sorted by the oracle."""
    x = inputs.splitmix64(r.seed, r.n)
    if r.key_type == "u64":
        keys, kmap = x.copy(), oracle.MAP_UNSIGNED
    else:
        low = (x & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        keys = low.view(np.float32).copy() if r.key_type == "f32" else low
        kmap = oracle.MAP_FLOAT if r.key_type == "f32" else oracle.MAP_UNSIGNED
    vals = np.arange(r.n, dtype=np.uint32) if r.has_payload else None
    oracle.stable_radix(keys, vals, key_map=kmap)
    return keys, vals


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_same_alone_and_in_the_mix(mode):
    require_gpu()
    torch = pytest.importorskip("torch")
    reqs = _mix()
    srv = serve.Server(budget_bytes=1 << 30, slots=3, mode=mode)
    st = srv.run(reqs, keep=lambda r: True, max_wall_s=120)
    assert st["done"] == len(reqs) and st["failed"] == 0 and st["rejected"] == 0
    if mode == "batched":
        assert st["mean_requests_per_launch"] > 1.0, st
    else:
        assert st["launches"] == len(reqs)
    for r in reqs:
        k, v = srv.kept[r.rid]
        ak, av = serve.sort_alone(r)
        assert torch.equal(k.view(torch.uint8), ak.view(torch.uint8)), r
        if r.has_payload:
            assert torch.equal(v, av), r
    for r in reqs[::9]:
        ek, ev = _host_reference(r)
        k, v = srv.kept[r.rid]
        assert same_bits(to_host(k), ek), r
        if r.has_payload:
            assert same_bits(to_host(v).view(np.uint32), ev), r


def test_budget_rejects_oversize_and_serves_the_rest():
    require_gpu()
    pytest.importorskip("torch")
    budget = 64 << 20
    reqs = [serve.Request(rid=0, n=1 << 22, key_type="u64", has_payload=True, seed=1),
            serve.Request(rid=1, n=5000, key_type="u32", has_payload=True, seed=2),
            serve.Request(rid=2, n=1 << 20, key_type="f32", has_payload=False, seed=3),
            serve.Request(rid=3, n=1 << 20, key_type="f32", has_payload=False, seed=4)]
    srv = serve.Server(budget_bytes=budget, slots=2, mode="batched")
    st = srv.run(reqs, keep=lambda r: True, max_wall_s=60)
    assert reqs[0].status == "rejected" and st["rejected"] == 1
    assert all(r.status == "done" for r in reqs[1:])
    assert st["peak_budget_bytes"] <= budget
    for r in reqs[1:]:
        ek, ev = _host_reference(r)
        k, v = srv.kept[r.rid]
        assert same_bits(to_host(k), ek)
        if r.has_payload:
            assert same_bits(to_host(v).view(np.uint32), ev)


def test_failed_launch_releases_its_slot_and_memory(monkeypatch):
    """A batch whose launch raises is marked failed; its stream slot and arena
    block come back and the other requests are still served."""
    require_gpu()
    torch = pytest.importorskip("torch")
    reqs = [serve.Request(rid=i, n=5000 + i, key_type="u32", has_payload=False, seed=i,
                          arrival_s=0.001 * i) for i in range(6)]
    srv = serve.Server(budget_bytes=64 << 20, slots=1, mode="plain")
    real = binding.sort_keys
    calls = {"n": 0}

    def flaky(*a, **k):
        calls["n"] += 1
        if calls["n"] == 3:
            # the batch's inputs are still being written on its stream (a
            # bounded spin stands in for a slow producer) when the launch fails
            torch.cuda._sleep(20_000_000)
            raise binding.BinarError(binding.ERR_INVALID_ARG, "test")
        return real(*a, **k)
    monkeypatch.setattr(binding, "sort_keys", flaky)
    real_release = srv.sched.release
    drained = []

    def release(b):   # a block comes back only once its stream has no work left
        drained.append(srv.streams[b.slot].query())
        real_release(b)
    monkeypatch.setattr(srv.sched, "release", release)
    st = srv.run(reqs, keep=lambda r: True, max_wall_s=60)
    assert drained and all(drained)
    assert st["failed"] == 1 and st["done"] == 5 and st["failed_launches"] == 1
    assert srv.arena.used == 0 and srv.free_slots == [0]
    failed = [r for r in reqs if r.status == "failed"]
    assert len(failed) == 1 and failed[0].error.startswith("launch:")
    for r in reqs:
        if r.status == "done":
            k, _ = srv.kept[r.rid]
            ak, _ = serve.sort_alone(r)
            assert torch.equal(k.view(torch.uint8), ak.view(torch.uint8))
