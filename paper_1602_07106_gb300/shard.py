"""Edge-range sharding across ranks (host logic).

Edge i is a pure function of (seed, n, d, n0, i) (paper section 2: the graph depends only on
the hash, not on the number of processors), so ranks need no exchange to generate edges:
each takes a contiguous slice of 0..m.  The streaming degree count (section 3) is the one
exchange: per-rank counters are summed.
"""
from __future__ import annotations


def strong_shard(m: int, rank: int, world: int) -> tuple[int, int]:
    """Slice of 0..m for `rank` when the whole graph is split over `world` ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank outside 0..world-1")
    return m * rank // world, m * (rank + 1) // world


def weak_shard(m_per_rank: int, rank: int) -> tuple[int, int]:
    """Slice of a graph world times larger: each rank keeps m_per_rank edges."""
    return rank * m_per_rank, (rank + 1) * m_per_rank


def sum_degree_counts(counts, group=None):
    """Sums per-rank degree counters in place (torch.distributed all-reduce)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts
