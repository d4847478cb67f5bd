"""Host-side partitioning of the work across GPUs (one process per GPU).

Points are independent (arXiv 2302.08381, Section 3: the call is parallel over
samples), so the path shards without any exchange: each rank evaluates its own
points into its own outputs. Only the timing is reduced (max over ranks). The
radial expansion (Eq. expansion) sums over the points of a centre; giving every
rank whole centres keeps that sum on one GPU, so it needs no collective either.
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


def centre_range(offsets, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [first, end) slice of whole centres for `rank`, balanced by
    points: rank r takes the centres whose first point lies in the r-th of
    `world` equal point ranges (CSR `offsets`, non-decreasing, offsets[0] = 0).
    A rank's point count differs from the even share by less than the largest
    centre."""
    import numpy as np

    offsets = np.asarray(offsets, dtype=np.int64)
    if offsets.ndim != 1 or offsets.size < 1 or offsets[0] != 0 or np.any(np.diff(offsets) < 0):
        raise ValueError("offsets must be a non-decreasing CSR array starting at 0")
    ncent = offsets.size - 1
    n_total = int(offsets[-1])
    starts = offsets[:-1]

    def first_centre(r: int) -> int:
        if r >= world:
            return ncent
        return int(np.searchsorted(starts, point_range(n_total, r, world)[0], side="left")) if r > 0 else 0

    if world <= 0 or not (0 <= rank < world):
        raise ValueError("bad partition arguments")
    return first_centre(rank), first_centre(rank + 1)


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
