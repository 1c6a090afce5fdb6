"""The multi-rank path of bench.py on CPU (gloo, world size 2): the slowest
rank's time is what every rank reports, launch counts add up over the
ranks, and the batch is shared out by LPT so that every graph goes to
exactly one rank."""
import itertools
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local = [3.5, 7.25][rank]
        got = bench.max_over_ranks(local, dist, "cpu")
        launches = bench.sum_over_ranks([9, 11][rank], dist, "cpu")
        sizes = [5, 1, 9, 3, 3, 8, 2]
        shard = bench.lpt_shards(sizes, world)[rank]
        out.put((rank, got, shard, launches))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_summed_launches_and_disjoint_shards():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [7.25, 7.25]
    assert [r[3] for r in res] == [20, 20]
    shards = [r[2] for r in res]
    assert sorted(itertools.chain(*shards)) == list(range(7))


def test_lpt_shards_balance():
    import bench
    sizes = [5, 1, 9, 3, 3, 8, 2]
    shards = bench.lpt_shards(sizes, 2)
    loads = [sum(sizes[i] for i in s) for s in shards]
    # LPT: largest first onto the lighter rank -> 9 | 8, 5 | 3, 3 | 2, 1
    assert shards == [[2, 3, 6], [0, 1, 4, 5]] or sorted(loads) == [15, 16]
    best = min(max(sum(sizes[i] for i in range(7) if m >> i & 1), sum(sizes[i] for i in range(7) if not m >> i & 1))
               for m in range(128))
    assert max(loads) <= 4 / 3 * best
    assert bench.lpt_shards(sizes, 1) == [list(range(7))]
    assert bench.lpt_shards([], 3) == [[], [], []]
