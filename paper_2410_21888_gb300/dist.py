"""Multi-rank execution of MBE3 batches: one process per GPU, fragments sharded by
greedy LPT on their 2mnk cost (largest first onto the least-loaded rank), no data-path
collective; the single exchange is an FP64 all-reduce of each rank's partial
sum_f c_f E_f.  The paper distributes polymers dynamically from a central queue
(Sec. "Overarching Algorithm"); with a static batch per time step, LPT gives the same
balance without a coordinator.
"""
from __future__ import annotations

import heapq

import numpy as np


def fragment_cost(o: int, v: int, X: int) -> float:
    return float(o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v ** 3
                 + 2 * o ** 3 * v * v)


def shard_lpt(costs, world: int):
    """Partition fragment indices over `world` ranks (list of index lists, each sorted)."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + costs[k], r))
    return [sorted(x) for x in out]


def imbalance(costs, shards) -> float:
    loads = [sum(costs[k] for k in s) for s in shards]
    return max(loads) / (sum(loads) / len(loads)) if sum(loads) > 0 else 1.0


def sharded_mbe3_total(energy_fn, frags, coeff, costs, rank: int, world: int, group=None):
    """This rank's share: energies of its fragments (energy_fn(list_of_frags) -> array),
    partial sum_f c_f E_f, then one all-reduce (math.fsum locally, FP64 across ranks)."""
    import math

    import torch
    import torch.distributed as dist

    mine = shard_lpt(costs, world)[rank]
    E = energy_fn([frags[k] for k in mine]) if mine else np.zeros(0)
    part = math.fsum(float(coeff[k]) * float(e) for k, e in zip(mine, E))
    t = torch.tensor([part], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), mine
