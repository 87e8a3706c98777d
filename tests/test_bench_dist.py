"""The multi-process timing of bench.py on CPU: two gloo ranks, each with its
own step time and unit count; the job rate takes the summed units over the
slowest rank's time, the same on every rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [1000.0, 2500.0][rank]
    units = [3_000_000_000, 5_000_000_000][rank]
    rate, job_ms, job_units = bench.job_rate(ms, units)
    out.put((rank, rate, job_ms, job_units))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, job_ms, job_units in res:
        assert job_ms == 2500.0
        assert job_units == 8_000_000_000
        assert rate == pytest.approx(8e9 / 2.5)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, job_ms, job_units = bench.job_rate(500.0, 1000)
    assert (rate, job_ms, job_units) == (2000.0, 500.0, 1000)
