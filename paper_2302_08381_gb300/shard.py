"""Host-side partitioning of the work across GPUs (one process per GPU).

Points are independent (arXiv 2302.08381, Section 3: the call is parallel over
samples), so the path shards without any exchange: each rank evaluates its own
points into its own outputs. Only the timing is reduced (max over ranks).
"""

from __future__ import annotations

import heapq


def point_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, end) slice of n_total points for `rank`; sizes differ by <= 1."""
    if world <= 0 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def set_bytes(n: int, l_max: int, gradients: bool = True, elem: int = 4) -> int:
    """HBM bytes one set moves: coordinates in, values (+ gradients) out."""
    k = (l_max + 1) ** 2
    return n * (3 * elem + k * elem * (4 if gradients else 1))


def balance_sets(sizes, lmaxes, world: int, gradients: bool = True):
    """Greedy longest-first assignment of whole sets to ranks by bytes moved.

    Returns a list (one per rank) of set indices. The largest set goes to the
    least-loaded rank first, which keeps the max load within the largest set
    of the optimum.
    """
    if world <= 0:
        raise ValueError("world must be positive")
    cost = [set_bytes(int(n), int(l), gradients) for n, l in zip(sizes, lmaxes)]
    order = sorted(range(len(cost)), key=lambda i: (-cost[i], i))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + cost[i], r))
    for r in range(world):
        out[r].sort()
    return out


def max_over_ranks(value: float, group=None) -> float:
    """Max of a per-rank float over the default process group (identity if
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
