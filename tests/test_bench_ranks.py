"""The replica path of bench.py across ranks, on CPU with gloo (world size 2): the job's time is its
slowest rank's and its throughput counts every rank's keys."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [40.0, 100.0][rank]  # rank 1 is the slow one
    value, ms = bench.job_throughput(local_ms, 1 << 20, 10, dist, torch.device("cpu"))
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_and_counts_all_keys():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = 2 * (1 << 20) * 10 / 0.1  # both ranks' keys over the slower rank's 100 ms
    for _, value, ms in got:
        assert ms == 100.0
        assert value == pytest.approx(want)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    value, ms = bench.job_throughput(50.0, 1000, 4)
    assert ms == 50.0 and value == pytest.approx(1000 * 4 / 0.05)
