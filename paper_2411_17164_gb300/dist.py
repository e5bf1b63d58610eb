"""Multi-rank host logic: halo partitions as data-parallel units (Sec. III-A).

Once every partition carries its halo, partitions are independent, so ranks
only exchange the parameter gradient once per step ("Gradient Aggregation":
the gradients of all partitions are summed before the update, which makes the
partitioned step equal to the full-graph step).  No activation exchange.

* ``assign_partitions`` balances partitions over ranks by their edge counts
  (each edge is one unit of message-passing work), deterministically.
* ``rank_batch`` keeps one rank's share of a graph's partitions: their ids
  are renumbered 0..k-1 and every other node is marked inner in no part, so
  ``xmgn.partition_halo`` builds exactly those partitions (with their halos).
* ``allreduce_gradient`` sums a gradient over ranks in rank order
  (all-gather, then a Neumaier-compensated fixed-order sum through the
  library's xmgn_grad_accumulate), so the result is bit-identical on every
  rank and from run to run, whatever the collective's internal order.
"""
from __future__ import annotations

import numpy as np
import torch


def assign_partitions(edge_counts, world: int):
    """Greedy longest-processing-time assignment: partitions sorted by edges
    (descending, ties by id) go to the least-loaded rank (ties by rank).
    Returns a list of partition-id lists, one per rank, each ascending."""
    order = sorted(range(len(edge_counts)), key=lambda p: (-int(edge_counts[p]), p))
    load = [0] * world
    out = [[] for _ in range(world)]
    for p in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(p)
        load[r] += int(edge_counts[p])
    return [sorted(x) for x in out]


def rank_batch(part, mine):
    """Part ids for one rank: the partitions listed in ``mine`` become
    0..len(mine)-1 (in that order), every other node -1 (inner in none of
    this rank's parts, so it can only appear in their halos)."""
    part = np.asarray(part)
    remap = np.full(int(part.max()) + 2 if part.size else 1, -1, dtype=np.int32)
    remap[np.asarray(mine, dtype=np.int64)] = np.arange(len(mine), dtype=np.int32)
    out = np.full(part.shape, -1, dtype=np.int32)
    ok = part >= 0
    out[ok] = remap[part[ok]]
    return out


def allreduce_gradient(grad: torch.Tensor, group=None, accumulate=None) -> torch.Tensor:
    """In-place sum of ``grad`` over all ranks of ``group``: every rank
    gathers all ranks' gradients and adds them in rank order with a
    compensated sum (the running error term is added at the end).
    ``accumulate(dst, src, comp)`` performs one compensated addition; it
    defaults to the library's xmgn_grad_accumulate (device tensors)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world == 1:
        return grad
    if accumulate is None:
        from paper_2411_17164_gb300 import xmgn
        accumulate = xmgn.grad_accumulate
    parts = [torch.empty_like(grad) for _ in range(world)]
    dist.all_gather(parts, grad.contiguous(), group=group)
    acc = parts[0].clone()
    comp = torch.zeros_like(acc)
    for p in parts[1:]:
        accumulate(acc, p, comp)
    accumulate(acc, comp)
    grad.copy_(acc)
    return grad
