"""bench.py's replica aggregation with two ranks over gloo on the CPU: every
rank gets the slowest rank's time and the whole-job value counts both ranks'
keys."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms_max = b.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms_max, b.replica_throughput(1000, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    times = [2.0, 5.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, times, out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, value = res[rank]
        assert ms_max == 5.0
        assert value == pytest.approx(2 * 1000 / 5e-3 / 1e9)


def test_single_process_passthrough():
    b = _bench()
    assert b.max_over_ranks(3.5, None, "cpu") == 3.5
    assert b.replica_throughput(256 << 20, 1, 6.0) == pytest.approx((256 << 20) / 6e-3 / 1e9)
