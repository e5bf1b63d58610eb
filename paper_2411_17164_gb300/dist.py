"""Multi-rank host logic: halo partitions as data-parallel units (Sec. III-A).

Once every partition carries its halo, partitions are independent, so ranks
only exchange the parameter gradient once per step ("Gradient Aggregation":
the gradients of all partitions are summed before the update, which makes the
partitioned step equal to the full-graph step).  No activation exchange.

* ``assign_partitions`` balances partitions over ranks by their edge counts
  (each edge is one unit of message-passing work), deterministically.
* ``allreduce_gradient`` sums a gradient tensor over ranks in rank order
  (all-gather, then a fixed-order sum), so the result is bit-identical on
  every rank and from run to run, whatever the collective's internal order.
"""
from __future__ import annotations

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


def allreduce_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of ``grad`` over all ranks of ``group``, in rank order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world == 1:
        return grad
    parts = [torch.empty_like(grad) for _ in range(world)]
    dist.all_gather(parts, grad.contiguous(), group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    grad.copy_(acc)
    return grad
