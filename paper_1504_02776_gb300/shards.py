"""Neutron-id shards of a multi-GPU run.

Rank r of w traces the ids first_id + [r n, (r + 1) n) of the same random stream (seed,
sim_id): weak scaling, with no exchange on the data path.  A neutron's history depends only
on (seed, sim_id, id), so the histograms and tallies of the ranks add up to those of one run
over the union of the ranges (up to the order of the FP64 additions).
"""
from __future__ import annotations


def shard(rank: int, world: int, n_per_rank: int, first_id: int = 0):
    """(first id, count) of `rank` when every rank traces n_per_rank neutrons."""
    if not (0 <= rank < world) or n_per_rank < 0 or first_id < 0:
        raise ValueError("bad shard request")
    return first_id + rank * n_per_rank, n_per_rank


def split(rank: int, world: int, n_total: int, first_id: int = 0):
    """(first id, count) of `rank` when n_total neutrons are divided over the ranks (strong
    scaling): contiguous ranges whose sizes differ by at most one."""
    if not (0 <= rank < world) or n_total < 0 or first_id < 0:
        raise ValueError("bad split request")
    lo = (n_total * rank) // world
    hi = (n_total * (rank + 1)) // world
    return first_id + lo, hi - lo
