"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process per GPU on a node).

The single solve runs as replicas (no collective on the data path); the batch of independent
instances is sharded over the ranks. Both report the largest rank time.
"""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist, torch.device("cpu"))
        mine = bench.shard(64, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (t, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_disjoint_shards():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for t, gathered in res.values():
        assert t == 2.5
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(64))                      # every instance exactly once
        assert set(gathered[0]).isdisjoint(gathered[1])


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, None) == 3.0
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
