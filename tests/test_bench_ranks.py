"""bench.py's multi-rank bookkeeping (replicas under torchrun) with two gloo ranks on the CPU:
the timed region's length is the slowest rank's, and the job's rate counts every rank's units."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _load_bench()
        local_ms = [1200.0, 1750.0][rank]           # the second rank is slower
        ms_max = bench.max_over_ranks(local_ms)
        dist.barrier()
        out[rank] = (ms_max, bench.job_rate(world, 5, ms_max / 1e3))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, rate = res[0]
    assert ms_max == 1750.0
    assert abs(rate - 2 * 5 / 1.75) < 1e-12


def test_single_process_needs_no_group():
    bench = _load_bench()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 4, 2.0) == 2.0
