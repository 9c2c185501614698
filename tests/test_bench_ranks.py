"""The benchmark's multi-rank combination (replicas: time = max over ranks, work = sum over
ranks) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 100 + 10 r ms for 192 site updates; end to end 2 + r s for 480 units
        res = bench.combine_ranks(dist, 100.0 + 10 * rank, 192.0, 2.0 + rank, 480.0, "cpu")
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_max_time_and_summed_work():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r] == (110.0, 384.0, 3.0, 960.0)


def test_single_process_passes_values_through():
    import bench
    assert bench.combine_ranks(None, 5.0, 7.0, 1.0, 9.0, "cpu") == (5.0, 7.0, 1.0, 9.0)
