"""The benchmark's multi-rank host logic with two gloo ranks on the CPU: the
whole-job timing (maximum of the ranks' timed regions) and work (sum), and
the round-robin split of a fixed set of LPs (every LP on exactly one rank).
The GPU ranks run the same functions over NCCL."""
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, w = bench.aggregate(dist, 10.0 + 5.0 * rank, 100 + rank, "cpu")
        mine = bench.shard(list(range(11)), rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, t, w, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_and_split():
    torch_mp = pytest.importorskip("torch.multiprocessing")
    ctx = torch_mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w, gathered in out:
        assert t == 15.0          # the slowest rank's time
        assert w == 201.0         # the work of both ranks
        flat = sorted(x for part in gathered for x in part)
        assert flat == list(range(11))
        assert not set(gathered[0]) & set(gathered[1])


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, 12.5, 7, "cpu") == (12.5, 7.0)
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]
