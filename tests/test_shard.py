"""CPU checks of the rank-range sharding (paper_2201_02460_gb300/shard.py):
range arithmetic, the exactness of the top-N merge, and the exchange itself
between two gloo processes on 127.0.0.1, with the oracle as each process's
range search."""
from __future__ import annotations

import math
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_02460_gb300 import shard
from tests.helpers import random_data

DT = np.dtype([("snp", "<u4", (8,)), ("mi", "<f8"), ("rank", "<u8")])


def _oracle_range(geno, pheno, k):
    n = geno.shape[0]

    def search(b, e, t):
        c, m, _ = O.search(geno, pheno, k, t, rank_begin=b, rank_end=e, with_counts=False)
        out = np.zeros(len(c), DT)
        for i in range(len(c)):
            out["snp"][i, :k] = c[i]
            out["mi"][i] = m[i]
            out["rank"][i] = O.rank(n, k, c[i])
        return out

    return search


def _full_topn(geno, pheno, k, t):
    n = geno.shape[0]
    c, m, _ = O.search(geno, pheno, k, t, with_counts=False)
    return [O.rank(n, k, x) for x in c], list(m)


@pytest.mark.parametrize("total,world", [(0, 1), (1, 3), (10, 3), (1000, 7), (2 ** 40 + 5, 8)])
def test_rank_ranges_partition(total, world):
    rr = shard.rank_ranges(total, world)
    assert len(rr) == world and rr[0][0] == 0 and rr[-1][1] == total
    assert all(rr[i][1] == rr[i + 1][0] for i in range(world - 1))
    sizes = [e - b for b, e in rr]
    assert max(sizes) - min(sizes) <= 1


def test_merge_of_range_topn_is_exact(oracle_lib):
    """The top-N of each of several ranges, merged, is the global top-N
    (duplicated SNPs force exact ties, broken by rank)."""
    geno, pheno = random_data(14, 300, seed=3)
    geno[9] = geno[2]
    k, t = 3, 30
    total = math.comb(14, k)
    search = _oracle_range(geno, pheno, k)
    for world in (2, 3, 7):
        parts = [search(b, e, t) for b, e in shard.rank_ranges(total, world)]
        got = shard.merge_topn(parts, t)
        want_r, want_m = _full_topn(geno, pheno, k, t)
        assert got["rank"].tolist() == want_r
        assert got["mi"].tolist() == want_m


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, k, t, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        geno, pheno = random_data(13, 257, seed=11)
        res = shard.sharded_search(_oracle_range(geno, pheno, k), math.comb(13, k), t)
        q.put((rank, res["rank"].tolist(), res["mi"].tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [3, 6])
def test_two_process_sharded_search(oracle_lib, k):
    """Two gloo processes each search half of the ranks and exchange their
    top-N: both end with the oracle's global top-N."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    t = 20
    procs = [ctx.Process(target=_worker, args=(r, 2, port, k, t, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            rank, ranks, mis = q.get(timeout=180)
            got[rank] = (ranks, mis)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    geno, pheno = random_data(13, 257, seed=11)
    want = _full_topn(geno, pheno, k, t)
    assert got[0] == got[1]
    assert got[0][0] == want[0] and got[0][1] == want[1]
