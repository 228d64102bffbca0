"""The replica path of bench.py (one process per GPU, no data exchange): the
timed region is the maximum over ranks and the rate counts every rank's work.
Run as two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, value = bench.whole_job([10.0, 30.0][rank], 1000.0, world, "cpu")
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_and_all_ranks_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 30.0
        assert value == pytest.approx(2 * 1000.0 / 0.030)


def test_whole_job_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job(20.0, 500.0, 1)
    assert ms == 20.0 and value == pytest.approx(500.0 / 0.020)
