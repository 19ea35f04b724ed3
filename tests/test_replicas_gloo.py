"""The bench's multi-GPU mode runs replicas (one join of the same workload per
rank, no data-path collective); the job's step time is the slowest rank's.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [5.0, 7.5][rank]
        q.put((rank, bench.slowest_rank_ms(mine, dist, "cpu"), bench.slowest_rank_ms(mine, None, "cpu")))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 7.5, 5.0), (1, 7.5, 7.5)]
