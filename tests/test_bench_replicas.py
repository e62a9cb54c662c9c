"""Host logic of the N > 1 (replica) path of bench.py on CPU: two gloo ranks
with different step times agree on the slowest time and the whole-job rate."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    ms = bench.max_over_ranks(ms_local, world, device="cpu")
    out[rank] = (ms, bench.job_throughput(ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_report_slowest_time_and_job_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, rate = res[0]
    assert ms == 150.0
    assert rate == pytest.approx(2 * 1e3 / 150.0)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(250.0, 1) == pytest.approx(4.0)
