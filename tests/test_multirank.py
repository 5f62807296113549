"""Multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2):
the step time is the maximum over ranks, the throughput counts every rank's
bits, and each rank decodes its own stream."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (r + 1) ms for the device step and (10 - r) ms end to end
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank], world, device="cpu")
        q.put((rank, got, bench.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, got, seed in res:
        assert got == [2.0, 10.0]
    assert len({seed for _, _, seed in res}) == world


def test_aggregate_counts_every_rank():
    one = bench.aggregate_gbps(1 << 24, 1, 0.3)
    assert bench.aggregate_gbps(1 << 24, 4, 0.3) == pytest.approx(4 * one)
    assert one == pytest.approx((1 << 24) / 0.3e-3 / 1e9)
    assert bench.max_over_ranks([1.5, 2], 1) == [1.5, 2.0]
