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


def test_centre_range_gives_whole_centres_balanced_by_points():
    import numpy as np

    rng = np.random.default_rng(7)
    for counts in (rng.integers(0, 80, 5000), np.zeros(10, np.int64), np.array([1000, 1, 1, 1]), np.array([], np.int64)):
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        n_total, big = int(offs[-1]), int(counts.max()) if counts.size else 0
        for world in (1, 2, 3, 8):
            ranges = [shard.centre_range(offs, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == counts.size
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            for a, b in ranges:
                assert abs(int(offs[b] - offs[a]) - n_total / world) <= big + 1
    with pytest.raises(ValueError):
        shard.centre_range(np.array([0, 5, 3]), 0, 2)


def _expansion_worker(rank, world, port, q):
    """Each rank expands its own whole centres (the oracle stands in for the
    kernel); the concatenation over ranks must equal the expansion of all
    centres, so no reduction of c is needed."""
    import numpy as np
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(8)
        counts = rng.integers(0, 12, 41)
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        xyz = inputs.shell_points(int(offs[-1]), 0.7, 3.0, seed=9).astype(np.float64)
        R = inputs.upstream(int(offs[-1]), 2 * 4, seed=10).reshape(-1, 2, 4).astype(np.float64)
        a, b = shard.centre_range(offs, rank, world)
        mine = oracle.expansion(xyz[offs[a]:offs[b]], R[offs[a]:offs[b]], offs[a:b + 1] - offs[a], 3)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        full = oracle.expansion(xyz, R, offs, 3)
        q.put((rank, float(np.abs(np.concatenate(parts) - full).max()), [p.shape[0] for p in parts]))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_expansion_by_whole_centres():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_expansion_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, sizes in res:
        assert err == 0.0 and sum(sizes) == 41 and min(sizes) > 0


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



def test_bench_launches_ranks_itself_dry_run():
    """bench.py --gpus 2 starts two ranks on its own (torch.distributed.run,
    gloo in the host-only dry run): both shard, barrier and reduce the max
    time, and rank 0 prints one line with n_gpus = 2."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                             "MASTER_PORT")}
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--steps", "5",
                          "--warmup", "3", "--n", "1000", "--dry-run"], capture_output=True, text=True, env=env,
                         timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(l) for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["dry_run"] and line["n_gpus"] == 2 and line["scaling"] == "weak"
    assert line["shards"] == [[0, 1000], [1000, 2000]]
    assert line["ms_per_step_max"] >= 2.0  # rank 1's stand-in steps (2 ms) set the max
