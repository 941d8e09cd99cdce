"""Parity at the workloads' full sizes and at the largest sample counts.

* Every contingency table of the tensor-core path (the counts of Section 2.2
  as an exact 0/1 product accumulated in FP32) against the oracle at the
  sample counts where the accumulator holds its largest values: 8192
  balanced samples (the order-4 workload), 16000 samples at case fractions
  0.3 and 0.7 (the largest datasets of the batched configuration), and about
  a million samples (counts near 2^18, the largest the API's exactness
  argument covers) with nearly monomorphic SNPs, so that single cells hold
  almost a whole class.
* The full-size order-3 and order-4 workloads, both counting paths (at
  order 3 both tensor-core variants), against
  the oracle's exhaustive top-N stored under tests/golden (written by
  tests/golden/make_fullsize.py, which calls only the oracle).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import brute
from oracle import oracle as O
from tests.golden import make_fullsize as G
from tests.helpers import F32_RTOL, F64_ATOL, check_topn, random_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_02460_gb300 import epi as E
    E.load()
    return E


@pytest.fixture(scope="module")
def ctx(epi):
    return epi.Context(0)


def _all_tables_exact(epi, ctx, geno, pheno, k):
    ds = epi.Dataset(ctx, geno, pheno)
    got = epi.debug_counts(ds, k)
    combs = np.array(brute.all_combinations(geno.shape[0], k), dtype=np.int32)
    want = O.tables(geno, pheno, combs)
    bad = np.nonzero((got != want).any(axis=(1, 2)))[0]
    assert len(bad) == 0, f"{len(bad)} of {len(combs)} tables differ, first ranks {bad[:5]}"
    return ds


@pytest.mark.parametrize("k,n,m,m1", [(3, 14, 8192, 4096), (4, 12, 8192, 4096), (3, 14, 16000, 4800),
                                      (3, 14, 16000, 11200), (4, 12, 16000, 4800), (5, 10, 16000, 11200)])
def test_tc_counts_bit_exact_large_k(epi, ctx, k, n, m, m1):
    geno, pheno = random_data(n, m, seed=9000 + 7 * k + m1, m1=m1)
    _all_tables_exact(epi, ctx, geno, pheno, k)


@pytest.mark.parametrize("k", [3, 4])
def test_tc_counts_bit_exact_largest_cells(epi, ctx, k):
    # about a million samples, three SNPs fixed at genotype 0 and the rest
    # nearly monomorphic: single cells hold up to a whole class (2^18 and
    # more), the accumulator's largest exact values
    m = (1 << 20) + 37
    m1 = int(0.3 * m)
    geno, pheno = random_data(8, m, seed=31 + k, m1=m1, p_levels=(0.005, 0.03))
    geno[:3] = 0
    _all_tables_exact(epi, ctx, geno, pheno, k)


def test_tc_search_large_k_unbalanced(epi, ctx):
    geno, pheno = random_data(40, 16000, seed=77, m1=4800)
    ds = epi.Dataset(ctx, geno, pheno)
    for k, top_n in ((3, 60), (4, 40)):
        r = epi.search(ds, k, top_n, path="tc")
        oc, om, ot = O.search(geno, pheno, k, top_n)
        check_topn(r.combs, r.mi, oc, om)
        assert (O.tables(geno, pheno, r.combs.astype(np.int32)) == r.counts).all()


def _golden_search(epi, ctx, name, paths):
    from paper_2201_02460_gb300 import synth
    if not os.path.exists(G.path_of(name)):
        pytest.fail(f"missing {G.path_of(name)}: run tests/golden/make_fullsize.py {name}")
    want = G.read(name)
    d, k, top_n = synth.make_workload(name)
    assert G.fingerprint(d.geno, d.pheno) == want["sha256"], "the synthetic generator changed"
    assert (k, top_n) == (want["order"], want["top_n"])
    ds = epi.Dataset(ctx, d.geno, d.pheno)
    m = d.n_samples
    for path in paths:
        # "tc_separate": the tensor path with separate case and control
        # accumulators (the combined-class variant is the default where it fits)
        ctx.set_tc_variant("separate" if path == "tc_separate" else "auto")
        try:
            r = epi.search(ds, k, top_n, path="tc" if path == "tc_separate" else path)
        finally:
            ctx.set_tc_variant("auto")
        check_topn(r.combs, r.mi, want["combs"], want["mi"])
        # every returned table is the oracle's table of that combination, and
        # both scores are those of the table
        t = O.tables(d.geno, d.pheno, r.combs.astype(np.int32))
        assert (t == r.counts).all(), path
        mi64 = np.array([O.mi(x[0], x[1], m) for x in t])
        np.testing.assert_allclose(r.mi, mi64, rtol=0, atol=F64_ATOL)
        assert (np.abs(r.mi_f32.astype(np.float64) - mi64) <= F32_RTOL * mi64 + 1e-12).all(), path
        # records equal to the stored ones wherever the order is unique
        same = [tuple(a) == tuple(b) for a, b in zip(r.combs.tolist(), want["combs"].tolist())]
        assert sum(same) >= len(same) - 2, path
    return d


def test_fullsize_order3_2000snp_4000_both_paths(epi, ctx):
    d = _golden_search(epi, ctx, "order3_2000snp_4000", ("tc", "tc_separate", "popc"))
    # the planted three-way parity (no marginal or pairwise effect) ranks first
    assert tuple(G.read("order3_2000snp_4000")["combs"][0]) == d.planted


def test_fullsize_order4_500snp_8192_both_paths(epi, ctx):
    _golden_search(epi, ctx, "order4_500snp_8192", ("tc", "popc"))
