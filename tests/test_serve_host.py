"""Host logic of the serving loop (no GPU): the arena that enforces the
device-memory budget and the scheduler's admission and batch formation."""
import random

import pytest

from paper_0811_3448_gb300.serve import (ALIGN, Arena, Request, Scheduler, block_layout,
                                         requests_from_mix)
from paper_0811_3448_gb300 import inputs


def fake_ws(n, kb, vb, segs):
    # shape of the real workspace: alternate buffers plus a per-segment part
    return 2 * n * (kb + vb) + 64 * segs + 4096


def test_arena_alignment_and_exhaustion():
    a = Arena(10 * ALIGN + 17)
    assert a.capacity == 10 * ALIGN
    offs = [a.alloc(1) for _ in range(10)]
    assert offs == [i * ALIGN for i in range(10)]
    assert a.alloc(1) is None
    a.free(offs[3])
    assert a.alloc(ALIGN + 1) is None           # one free unit only
    assert a.alloc(ALIGN) == offs[3]


def test_arena_coalesces_against_a_model():
    """Random alloc/free against a byte-map model: no overlap, full coalescing
    (after freeing everything there is one free range again)."""
    rng = random.Random(7)
    cap = 1000 * ALIGN
    a = Arena(cap)
    owner = [None] * (cap // ALIGN)
    live = {}
    for step in range(5000):
        if live and rng.random() < 0.45:
            off = rng.choice(sorted(live))
            size = live.pop(off)
            for u in range(off // ALIGN, (off + size) // ALIGN):
                assert owner[u] == off
                owner[u] = None
            a.free(off)
        else:
            want = rng.randint(1, 40 * ALIGN)
            off = a.alloc(want)
            size = -(-want // ALIGN) * ALIGN
            # first fit: None exactly when no run of free units is long enough
            run, best, first = 0, 0, None
            for u, o in enumerate(owner):
                run = run + 1 if o is None else 0
                best = max(best, run)
                if first is None and run * ALIGN >= size:
                    first = (u - run + 1) * ALIGN
            if off is None:
                assert best * ALIGN < size
                continue
            assert off == first
            for u in range(off // ALIGN, (off + size) // ALIGN):
                assert owner[u] is None
                owner[u] = off
            live[off] = size
        assert a.used == sum(live.values())
    for off in list(live):
        a.free(off)
    assert a.free_list == [(0, cap)] and a.used == 0


def test_arena_double_free_raises():
    a = Arena(4 * ALIGN)
    off = a.alloc(10)
    a.free(off)
    with pytest.raises(KeyError):
        a.free(off)


def test_block_layout_alignment():
    L = block_layout([1000, 7, 3], 8, 4, fake_ws)
    assert L.n == 1010
    for off in (L.keys_off, L.vals_off, L.offs_off, L.ws_off, L.total):
        assert off % ALIGN == 0
    assert L.vals_off >= 1010 * 8 and L.offs_off >= L.vals_off + 1010 * 4
    assert L.ws_off >= L.offs_off + 4 * 8 and L.total >= L.ws_off + L.ws_bytes


def _req(rid, n, kt="u32", p=False, t=0.0):
    return Request(rid=rid, n=n, key_type=kt, has_payload=p, seed=rid, arrival_s=t)


def test_oversize_request_rejected_others_served():
    a = Arena(1 << 20)
    s = Scheduler(a, fake_ws)
    big = _req(0, 1 << 20, "u64", True)
    assert not s.submit(big) and big.status == "rejected" and big.error
    small = _req(1, 1000)
    assert s.submit(small)
    b = s.next_batch()
    assert b.requests == [small] and b.starts == [0, 1000]
    s.release(b)
    assert s.next_batch() is None and a.used == 0


def test_batches_group_by_class_in_arrival_order():
    a = Arena(1 << 30)
    s = Scheduler(a, fake_ws)
    rs = [_req(0, 100, "u32"), _req(1, 200, "u64"), _req(2, 300, "u32"),
          _req(3, 400, "u32", True), _req(4, 500, "u32")]
    for r in rs:
        s.submit(r)
    b1 = s.next_batch()
    assert [r.rid for r in b1.requests] == [0, 2, 4] and b1.starts == [0, 100, 400, 900]
    b2 = s.next_batch()
    assert [r.rid for r in b2.requests] == [1]
    b3 = s.next_batch()
    assert [r.rid for r in b3.requests] == [3]
    assert s.next_batch() is None
    # blocks do not overlap
    spans = sorted((b.arena_off, b.arena_off + b.layout.total) for b in (b1, b2, b3))
    assert all(x[1] <= y[0] for x, y in zip(spans, spans[1:]))


def test_head_waits_for_memory_without_overtaking():
    need = block_layout([5000], 4, 0, fake_ws).total
    a = Arena(need + need // 2)
    s = Scheduler(a, fake_ws)
    s.submit(_req(0, 5000))
    b0 = s.next_batch()
    s.submit(_req(1, 5000))       # does not fit until b0 is released
    s.submit(_req(2, 10, "u64"))  # would fit, but must not overtake request 1
    assert s.next_batch() is None
    s.release(b0)
    b1 = s.next_batch()
    assert [r.rid for r in b1.requests] == [1]
    b2 = s.next_batch()
    assert [r.rid for r in b2.requests] == [2]


def test_batch_limits():
    a = Arena(1 << 30)
    s = Scheduler(a, fake_ws, max_batch_keys=1000, max_batch_requests=3)
    for i in range(6):
        s.submit(_req(i, 300))
    sizes = []
    while (b := s.next_batch()) is not None:
        sizes.append(len(b.requests))
        assert b.layout.n <= 1000
    assert sizes == [3, 3]
    s2 = Scheduler(Arena(1 << 30), fake_ws, max_batch_keys=1000)
    s2.submit(_req(0, 5000))      # one request above the key cap still runs alone
    assert s2.next_batch().layout.n == 5000


def test_simulated_run_drains_without_deadlock():
    """Discrete-event run of the scheduler with a fake device (service time
    proportional to keys), tight budget, 3 slots: every admitted request
    completes and the budget is never exceeded."""
    mix = inputs.config5_requests(rate_hz=2000.0, duration_s=0.05, min_log2=10, span_log2=10)
    reqs = requests_from_mix(mix)
    budget = 8 * block_layout([1 << 20], 8, 4, fake_ws).total
    a = Arena(budget)
    s = Scheduler(a, fake_ws, max_batch_keys=1 << 21)
    slots, inflight, t, i = 3, [], 0.0, 0
    while i < len(reqs) or s.queued or inflight:
        nxt = [reqs[i].arrival_s] if i < len(reqs) else []
        nxt += [d for d, _ in inflight]
        t = max(t, min(nxt))
        while i < len(reqs) and reqs[i].arrival_s <= t:
            s.submit(reqs[i])
            i += 1
        for d, b in list(inflight):
            if d <= t:
                inflight.remove((d, b))
                for r in b.requests:
                    r.status, r.t_done = "done", d
                s.release(b)
        while len(inflight) < slots and (b := s.next_batch()) is not None:
            assert a.used <= a.capacity
            inflight.append((t + 1e-9 * b.layout.n + 5e-6, b))
    assert all(r.status == "done" for r in reqs)
    assert a.used == 0 and a.peak <= budget


def test_long_backlog_batches_in_constant_time_per_request():
    """A backlog of 200,000 queued requests is drained one request per batch
    without quadratic work (the plain form under overload)."""
    import time
    a = Arena(1 << 40)
    s = Scheduler(a, fake_ws, max_batch_requests=1)
    for i in range(200_000):
        s.submit(_req(i, 1000, ("u32", "u64", "f32")[i % 3], bool(i & 1)))
    t0 = time.perf_counter()
    order = []
    while (b := s.next_batch()) is not None:
        order.append(b.requests[0].rid)
        s.release(b)
    assert order == list(range(200_000))           # oldest first across classes
    assert time.perf_counter() - t0 < 30.0


def test_linger_waits_only_for_small_young_batches():
    """A batch lingers while its class holds fewer than linger_keys queued
    keys and its oldest request is younger than linger_s; never otherwise."""
    arena = Arena(1 << 30)
    sched = Scheduler(arena, fake_ws)
    assert not sched.should_linger(0.0, 1e-3, 1 << 20)              # nothing queued
    sched.submit(Request(rid=0, n=1000, key_type="u32", has_payload=False, seed=0,
                               arrival_s=1.0))
    assert sched.should_linger(1.0002, 1e-3, 1 << 20)                # small and young
    assert not sched.should_linger(1.002, 1e-3, 1 << 20)             # waited long enough
    sched.submit(Request(rid=1, n=2 << 20, key_type="u32", has_payload=False, seed=1,
                               arrival_s=1.0001))
    assert not sched.should_linger(1.0002, 1e-3, 1 << 20)            # class already large
    b = sched.next_batch()
    assert [r.rid for r in b.requests] == [0, 1]
