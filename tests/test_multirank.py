"""The benchmark's multi-rank host logic with two gloo ranks on the CPU: the
whole-job timing (maximum of the ranks' timed regions) and work (sum), the
round-robin and longest-processing-time-first splits of a fixed set of LPs
(every LP on exactly one rank, the LPT makespan within Graham's 4/3 bound of
the brute-forced optimum), and per-rank reports gathered back into the whole
batch's order.  The GPU ranks run the same functions over NCCL.  (Not run
on GPUs: every run of this build used one GPU.)"""
import itertools
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    import lpgen
    return [lpgen.batch_lp(i, m_range=(50, 400)) for i in range(12)]


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
        # the LPT split of a batch, each rank "solving" its LPs (a stand-in
        # report per LP), the reports gathered back into the batch's order
        lps = _batch()
        weights = [bench.lp_weight(lp) for lp in lps]
        idx = bench.lpt_partition(weights, world)[rank]
        reps = [(k, {"lp": k, "iters": 10 * k + 1}) for k in idx]
        all_reps = [None] * world
        dist.all_gather_object(all_reps, reps)
        merged = dict(kv for part in all_reps for kv in part)
        q.put((rank, t, w, gathered, idx, [merged[k] for k in range(len(lps))]))
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
    import bench
    lps = _batch()
    weights = [bench.lp_weight(lp) for lp in lps]
    parts = {}
    for rank, t, w, gathered, idx, reports in out:
        assert t == 15.0          # the slowest rank's time
        assert w == 201.0         # the work of both ranks
        flat = sorted(x for part in gathered for x in part)
        assert flat == list(range(11))
        assert not set(gathered[0]) & set(gathered[1])
        parts[rank] = idx
        # every LP's report is back, in the batch's order
        assert [r["lp"] for r in reports] == list(range(len(lps)))
        assert all(r["iters"] == 10 * k + 1 for k, r in enumerate(reports))
    # each LP on exactly one rank
    assert sorted(parts[0] + parts[1]) == list(range(len(lps)))
    assert not set(parts[0]) & set(parts[1])
    # makespan within Graham's bound of the brute-forced optimum
    make = max(sum(weights[k] for k in parts[r]) for r in (0, 1))
    opt = min(max(sum(w_ for w_, b in zip(weights, bits) if b), sum(w_ for w_, b in zip(weights, bits) if not b))
              for bits in itertools.product((0, 1), repeat=len(weights)))
    assert make <= (4.0 / 3.0 - 1.0 / 6.0) * opt + 1e-9


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, 12.5, 7, "cpu") == (12.5, 7.0)
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]


def test_lpt_partition_known_cases():
    import bench
    # Graham's tight example for 2 bins: 3, 3, 2, 2, 2 -> LPT 7 against the optimum 6
    parts = bench.lpt_partition([3, 3, 2, 2, 2], 2)
    loads = sorted(sum([3, 3, 2, 2, 2][k] for k in p) for p in parts)
    assert loads == [5, 7]
    # equal weights spread evenly; one bin takes everything
    assert [len(p) for p in bench.lpt_partition([1.0] * 10, 4)] == [3, 3, 2, 2]
    assert bench.lpt_partition([5, 1, 2], 1) == [[0, 1, 2]]
    # the largest item goes first, to bin 0
    assert 0 in bench.lpt_partition([9, 1, 1, 1], 2)[0]
