"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""

import os
import socket


import pytest
import torch.multiprocessing as mp

from paper_2302_08381_gb300 import inputs, shard


def test_point_range_partitions_exactly():
    for n in (0, 1, 7, 1000, 4_194_304):
        for world in (1, 2, 3, 8):
            ranges = [shard.point_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.point_range(10, 2, 2)


def test_balance_sets_covers_and_balances():
    sizes, lmax, _ = inputs.ragged_sets(512, [3, 6, 8, 12], 1000, 200_000, seed=5)
    for world in (1, 2, 4, 8):
        parts = shard.balance_sets(sizes, lmax, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [sum(shard.set_bytes(sizes[i], lmax[i]) for i in p) for p in parts]
        biggest = max(shard.set_bytes(n, l) for n, l in zip(sizes, lmax))
        assert max(loads) - min(loads) <= biggest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 1001
        a, b = shard.point_range(n, rank, world)
        got = dist_gather_ranges(dist, a, b, world)
        t = shard.max_over_ranks(float(rank + 1) * 0.5)
        sizes, lmax, _ = inputs.ragged_sets(64, [3, 6, 8, 12], 10, 1000, seed=6)
        mine = shard.balance_sets(sizes, lmax, world)[rank]
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        q.put((rank, got, t, sorted(i for p in everyone for i in p)))
    finally:
        dist.destroy_process_group()


def dist_gather_ranges(dist, a, b, world):
    out = [None] * world
    dist.all_gather_object(out, (a, b))
    return out


def test_two_rank_gloo_sharding_and_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ranges, t, sets in res:
        assert ranges == [(0, 501), (501, 1001)]
        assert t == 1.0  # max over ranks of 0.5 * (rank + 1)
        assert sets == list(range(64))

