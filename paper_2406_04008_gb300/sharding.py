"""Placement of independent collages on ranks (one process per GPU).

Collages share nothing on the data path, so a batch splits across GPUs by whole collages with no
collective: every rank runs its share in one batched handle.  The split balances an estimate of
the per-iteration work (pixels of the finest grid plus a term per element) with the greedy
longest-processing-time rule, deterministically, so all ranks compute the same assignment without
communicating.
"""
from __future__ import annotations


def work_estimate(problem: dict) -> float:
    """Relative per-iteration cost of one collage: its pixels plus 1024 pixel-equivalents per
    element (the per-element binning and raster overhead)."""
    grid = int(problem.get("grid", 0)) or 1024
    return float(grid) * grid + 1024.0 * len(problem["kind"])


def assign(weights, world: int):
    """Greedy LPT: heaviest first onto the least-loaded rank (ties: lower rank, lower index).
    Returns (owner per item, load per rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    loads = [0.0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        owner[i] = r
        loads[r] += weights[i]
    return owner, loads


def shard(problems, world: int, rank: int):
    """Indices of the collages rank `rank` runs, in their original order."""
    owner, _ = assign([work_estimate(p) for p in problems], world)
    return [i for i, o in enumerate(owner) if o == rank]
