"""Placement of independent piles on several GPUs (one process per GPU).

Piles never interact, so sharding needs no data-path collective: each rank
owns a subset of piles and steps them in its own world.  The cost of a pile's
step is dominated by its direct-sum gravity, ~N_p^2, plus the O(N_p) contact
and bookkeeping work; piles are assigned largest first to the least-loaded
rank (LPT greedy), which keeps the most expensive rank within 4/3 of optimal.
"""
from __future__ import annotations


def pile_cost(n_spheres: int, linear_weight: float = 2000.0) -> float:
    """Relative step cost of a pile of n spheres."""
    return float(n_spheres) ** 2 + linear_weight * float(n_spheres)


def shard_piles(sizes, world_size: int):
    """Deterministic assignment: returns one list of pile indices per rank."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-pile_cost(sizes[k]), k))
    load = [0.0] * world_size
    out = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += pile_cost(sizes[k])
    for lst in out:
        lst.sort()
    return out


def imbalance(sizes, shards) -> float:
    """Most loaded rank's cost over the mean cost (1.0 = perfect)."""
    loads = [sum(pile_cost(sizes[k]) for k in s) for s in shards]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0
