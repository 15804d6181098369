"""Sharding the components of one combination over ranks (one GPU per rank).

The components of Eq. (19) are independent problems and the combination is
linear in them, so a multi-GPU run gives each rank a subset of components,
solves and combines only those (st_combine_subset), and sums the partial
target arrays with one collective.  The partition balances an estimate of
each component's cost (its space-time unknowns) by the longest-processing-
time rule: components in decreasing cost, each to the least-loaded rank.
"""
from __future__ import annotations

from typing import List, Sequence


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Component indices per rank (LPT greedy; ties to the lower rank and the
    lower component index, so every rank computes the same partition)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(k)
        load[r] += float(costs[k])
    return [sorted(p) for p in parts]


def component_costs(solver) -> List[float]:
    """Cost estimate per component: its space-time unknowns."""
    return [float(ci.n_space * ci.n_time) for ci in solver.components()]


def sharded_combine(solver, jx_star: int, jt_star: int, out, rank: int, world: int, group=None):
    """Solve this rank's components, write their part of u^CF into out (a
    device tensor of the target shape) and sum the parts over the process
    group (all-reduce), so that every rank ends with the full u^CF."""
    import torch.distributed as dist
    mine = partition(component_costs(solver), world)[rank]
    for k in mine:
        solver.solve(k, sync=False)
    if mine:
        solver.combine_subset(jx_star, jt_star, mine, out)
    else:
        out.zero_()
    if world > 1:
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
