"""Rank-range sharding of one exhaustive search over several processes.

Every k-combination costs the same (Section 2.2: 3^k cells over all
individuals), so the lexicographic rank space [0, C(n, k)) is split into
contiguous ranges of near-equal size, one per process (one GPU each).  Each
process searches its range (``epi.search(..., rank_range=...)``, the C-ABI's
epi_search_range) and keeps its top-N; the per-range top-N records are then
gathered and merged by (MI desc, rank asc).  The merge is exact: every member
of the global top-N is in the top-N of its own range.  Gathering the records
is the only exchange between processes.

The search of a range is passed in as a function, so the same code serves
the GPU path and a CPU check of the exchange.
"""
from __future__ import annotations

import numpy as np


def rank_ranges(total: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) ranges covering [0, total), sizes differing by
    at most one."""
    if world < 1 or total < 0:
        raise ValueError("need world >= 1 and total >= 0")
    base, extra = divmod(total, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def merge_topn(parts, top_n: int) -> np.ndarray:
    """The best top_n records of several record arrays (fields "mi" and
    "rank"), by (mi desc, rank asc)."""
    parts = list(parts)
    if not parts:
        raise ValueError("no record arrays to merge")
    allr = np.concatenate(parts)
    order = np.lexsort((allr["rank"], -allr["mi"]))
    return allr[order[:top_n]]


def sharded_search(search_range, total: int, top_n: int, group=None) -> np.ndarray:
    """This process's share of the search and the merged global top-N.

    search_range(begin, end, top_n) returns the top-N records of ranks
    [begin, end).  With torch.distributed initialised, every rank searches
    its range and all ranks receive the merged result; without it the whole
    range is searched here."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return merge_topn([search_range(0, total, top_n)], top_n)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    b, e = rank_ranges(total, world)[rank]
    mine = search_range(b, e, top_n) if e > b else None
    gathered = [None] * world
    dist.all_gather_object(gathered, mine, group=group)
    return merge_topn([g for g in gathered if g is not None], top_n)
