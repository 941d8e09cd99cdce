"""Pins of the CPU oracle against facts fixed outside it.

Each test ties one part of the oracle to something it does not compute
itself: the printed worked example of Fig. 2, the combination counts of
Table 2, a per-individual brute-force counter, library routines (scipy's
G-test, scikit-learn's mutual information), closed forms, invariants of
Eq. 1-3, and brute-force enumeration with itertools.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

from oracle import brute
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Fig. 2 worked example
# ----------------------------------------------------------------------------

def _fig2():
    snps, comb, misprint = {}, {}, None
    with open(os.path.join(GOLDEN, "fig2_genotype_tables.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            if p[0] == "snp":
                snps.setdefault(p[1], {})[int(p[2])] = (p[3], p[4])
            elif p[0] == "comb":
                comb[p[2]] = (p[3], p[4])
            elif p[0] == "misprint":
                misprint = dict(row=p[2], controls=p[4], equals=p[6])
    return snps, comb, misprint


def _bits_to_int(s: str) -> int:
    """Drawing order (leftmost = individual 0) to LSB-first integer."""
    return sum(1 << b for b, ch in enumerate(s) if ch == "1")


def _fig2_dataset():
    snps, _, _ = _fig2()
    geno = np.zeros((2, 32), dtype=np.uint8)
    pheno = np.array([1] * 16 + [0] * 16, dtype=np.uint8)
    for s_idx, name in enumerate(("i", "j")):
        for half in (0, 1):
            for b in range(16):
                rows = [r for r in (1, 2, 3) if snps[name][r][half][b] == "1"]
                assert len(rows) == 1, "each individual has exactly one genotype"
                geno[s_idx, half * 16 + b] = rows[0] - 1
    return geno, pheno


def test_fig2_tables_are_partitions():
    snps, _, _ = _fig2()
    for name in ("i", "j"):
        for half in (0, 1):
            rows = [_bits_to_int(snps[name][r][half]) for r in (1, 2, 3)]
            assert rows[0] & rows[1] == 0 and rows[0] & rows[2] == 0 and rows[1] & rows[2] == 0
            assert rows[0] | rows[1] | rows[2] == 0xFFFF


def test_fig2_single_snp_tables(oracle_lib):
    snps, _, _ = _fig2()
    geno, pheno = _fig2_dataset()
    for s_idx, name in enumerate(("i", "j")):
        case, ctrl = O.genotype_table(geno, pheno, (s_idx,))
        assert case.shape == (3, 1) and ctrl.shape == (3, 1)
        for r in (1, 2, 3):
            assert int(case[r - 1, 0]) == _bits_to_int(snps[name][r][0])
            assert int(ctrl[r - 1, 0]) == _bits_to_int(snps[name][r][1])


def test_fig2_combined_rows(oracle_lib):
    snps, comb, mis = _fig2()
    geno, pheno = _fig2_dataset()
    case, ctrl = O.genotype_table(geno, pheno, (0, 1))
    assert case.shape == (9, 1)
    for label, (c_bits, n_bits) in comb.items():
        ri, rj = int(label[0]), int(label[1])
        row = (ri - 1) * 3 + (rj - 1)
        assert int(case[row, 0]) == _bits_to_int(c_bits), label
        if label == mis["row"]:
            # the printed control half is the figure's misprint
            assert int(ctrl[row, 0]) == _bits_to_int(mis["controls"])
            e = mis["equals"]
            other = (int(e[0]) - 1) * 3 + (int(e[1]) - 1)
            assert int(ctrl[other, 0]) == _bits_to_int(n_bits)
        else:
            assert int(ctrl[row, 0]) == _bits_to_int(n_bits), label
    # every row is the AND of the printed single-SNP rows
    for ri in (1, 2, 3):
        for rj in (1, 2, 3):
            row = (ri - 1) * 3 + (rj - 1)
            for half, got in ((0, case), (1, ctrl)):
                want = _bits_to_int(snps["i"][ri][half]) & _bits_to_int(snps["j"][rj][half])
                assert int(got[row, 0]) == want


def test_fig2_contingency_and_mi(oracle_lib):
    sk = pytest.importorskip("sklearn.metrics")
    geno, pheno = _fig2_dataset()
    t = O.tables(geno, pheno, [[0, 1]])[0]
    assert t.tolist() == brute.table(geno, pheno, (0, 1)).tolist()
    assert t.sum(axis=1).tolist() == [16, 16]
    mi_o = O.mi(t[0], t[1], 32)
    x = 3 * geno[0].astype(int) + geno[1]
    assert mi_o == pytest.approx(sk.mutual_info_score(pheno, x), rel=1e-12, abs=1e-15)
    # the value implied by the printed tables (nats)
    assert mi_o == pytest.approx(0.0872029308616535, rel=1e-12)


# ----------------------------------------------------------------------------
# Table 2 combination counts and enumeration
# ----------------------------------------------------------------------------

def test_table2_counts(oracle_lib):
    assert O.binom(25000, 2) == 312487500
    assert O.binom(25000, 2) * 9 == 2812387500
    # the row printed for order 4 says 242 SNPs, but its combinations and
    # cells are those of 171 SNPs
    assert O.binom(171, 4) == 34389810
    assert O.binom(171, 4) * 81 == 2785574610
    assert O.binom(242, 4) != 34389810
    assert O.binom(23, 8) == 490314
    assert O.binom(23, 8) * 6561 == 3216950154


def test_binom_matches_math(oracle_lib):
    for n in (0, 1, 5, 31, 200, 2000, 100000):
        for k in range(0, 9):
            want = math.comb(n, k)
            # values beyond 64 bits come back as the UINT64_MAX sentinel
            assert O.binom(n, k) == (want if want < 2 ** 64 else 2 ** 64 - 1)


@pytest.mark.parametrize("n,k", [(1, 1), (5, 1), (6, 2), (9, 3), (10, 4), (11, 5), (12, 6), (10, 8)])
def test_unrank_is_lexicographic(oracle_lib, n, k):
    combs = list(itertools.combinations(range(n), k))
    for r, c in enumerate(combs):
        assert O.unrank(n, k, r) == c
        assert O.rank(n, k, c) == r


def test_rank_large(oracle_lib):
    n, k = 2000, 3
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = tuple(sorted(rng.choice(n, size=k, replace=False).tolist()))
        r = O.rank(n, k, c)
        assert O.unrank(n, k, r) == c
    assert O.unrank(n, k, O.binom(n, k) - 1) == (1997, 1998, 1999)


# ----------------------------------------------------------------------------
# contingency tables against the per-individual brute force
# ----------------------------------------------------------------------------

def _rand(n, m, seed, m1=None):
    rng = np.random.default_rng(seed)
    geno = rng.integers(0, 3, size=(n, m), dtype=np.uint8)
    if m1 is None:
        pheno = rng.integers(0, 2, size=m, dtype=np.uint8)
    else:
        pheno = np.zeros(m, np.uint8)
        pheno[rng.choice(m, size=m1, replace=False)] = 1
    return geno, pheno


@pytest.mark.parametrize("m", [1, 7, 31, 32, 33, 63, 64, 65, 70, 129])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tables_match_brute_force(oracle_lib, k, m):
    n = 9
    geno, pheno = _rand(n, m, seed=1000 * k + m)
    combs = brute.all_combinations(n, k)
    got = O.tables(geno, pheno, combs)
    for c, t in zip(combs, got):
        assert t.tolist() == brute.table(geno, pheno, c).tolist(), c


@pytest.mark.parametrize("m1", [0, 1, 40])
def test_tables_single_class(oracle_lib, m1):
    geno, pheno = _rand(7, 40, seed=3, m1=m1)
    combs = brute.all_combinations(7, 3)
    got = O.tables(geno, pheno, combs)
    for c, t in zip(combs, got):
        assert t.tolist() == brute.table(geno, pheno, c).tolist()


def test_table_invariants(oracle_lib):
    n, m, k = 8, 101, 4
    geno, pheno = _rand(n, m, seed=11)
    m1 = int(pheno.sum())
    for c in brute.all_combinations(n, k):
        t = O.tables(geno, pheno, [c])[0].astype(np.int64)
        assert t[0].sum() == m1 and t[1].sum() == m - m1
        # summing out SNP position d gives the table of the remaining SNPs
        for d in range(k):
            rest = tuple(s for i, s in enumerate(c) if i != d)
            marg = t.reshape(2, *([3] * k)).sum(axis=1 + d).reshape(2, -1)
            assert marg.tolist() == O.tables(geno, pheno, [rest])[0].astype(np.int64).tolist()
    # order 1: the table is the per-SNP genotype count per class
    for s in range(n):
        t = O.tables(geno, pheno, [[s]])[0]
        for g in range(3):
            assert t[0, g] == int(((geno[s] == g) & (pheno == 1)).sum())
            assert t[1, g] == int(((geno[s] == g) & (pheno == 0)).sum())


def test_invalid_inputs_rejected(oracle_lib):
    geno, pheno = _rand(5, 10, seed=2)
    with pytest.raises(ValueError):
        O.tables(geno, pheno, [[1, 1]])
    with pytest.raises(ValueError):
        O.tables(geno, pheno, [[2, 1]])
    bad = geno.copy()
    bad[0, 0] = 3
    with pytest.raises(ValueError):
        O.tables(bad, pheno, [[0, 1]])
    badp = pheno.copy()
    badp[0] = 2
    with pytest.raises(ValueError):
        O.tables(geno, badp, [[0, 1]])


# ----------------------------------------------------------------------------
# mutual information (Eq. 1-3)
# ----------------------------------------------------------------------------

def test_mi_against_scipy_g_test(oracle_lib):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    for trial in range(200):
        cells = 3 ** int(rng.integers(1, 5))
        t = rng.integers(0, 30, size=(2, cells))
        t[:, rng.random(cells) < 0.2] = 0
        keep = t.sum(axis=0) > 0
        if t[0].sum() == 0 or t[1].sum() == 0 or keep.sum() < 2:
            continue
        m = int(t.sum())
        g, *_ = stats.chi2_contingency(t[:, keep], correction=False, lambda_="log-likelihood")
        assert O.mi(t[0], t[1], m) == pytest.approx(g / (2 * m), rel=1e-10, abs=1e-14)


def test_mi_against_sklearn(oracle_lib):
    sk = pytest.importorskip("sklearn.metrics")
    geno, pheno = _rand(6, 97, seed=21)
    for c in brute.all_combinations(6, 3):
        t = O.tables(geno, pheno, [c])[0]
        x = (9 * geno[c[0]].astype(int) + 3 * geno[c[1]] + geno[c[2]])
        assert O.mi(t[0], t[1], 97) == pytest.approx(sk.mutual_info_score(pheno, x), rel=1e-11, abs=1e-15)


def test_mi_closed_forms(oracle_lib):
    # perfectly separating table with balanced classes: MI = H(Y) = ln 2
    assert O.mi([10, 0, 0], [0, 10, 0], 20) == pytest.approx(math.log(2), rel=1e-15)
    # unbalanced perfect separation: MI = H(Y)
    hy = -(0.25 * math.log(0.25) + 0.75 * math.log(0.75))
    assert O.mi([5, 0, 0, 0], [0, 7, 8, 0], 20) == pytest.approx(hy, rel=1e-14)
    # exactly factorised tables: MI = 0
    assert abs(O.mi([4, 8, 2, 6], [6, 12, 3, 9], 50)) < 1e-15
    assert abs(O.mi([3, 3, 3], [3, 3, 3], 18)) < 1e-15
    # one class only: MI = 0 exactly
    assert O.mi([0, 0, 0], [5, 2, 9], 16) == 0.0
    # a single occupied cell: MI = 0
    assert O.mi([0, 4, 0], [0, 9, 0], 13) == pytest.approx(0.0, abs=1e-15)


def test_mi_bounds_symmetry_and_chain_rule(oracle_lib):
    n, m = 7, 83
    geno, pheno = _rand(n, m, seed=31)
    m1 = int(pheno.sum())
    hy = -sum(p * math.log(p) for p in (m1 / m, 1 - m1 / m) if p > 0)
    mi_of = {}
    for k in (1, 2, 3, 4):
        for c in brute.all_combinations(n, k):
            t = O.tables(geno, pheno, [c])[0]
            v = O.mi(t[0], t[1], m)
            px = (t[0] + t[1]) / m
            hx = -sum(p * math.log(p) for p in px if p > 0)
            assert -1e-15 <= v <= min(hx, hy) + 1e-12
            mi_of[c] = v
            # the same table under any SNP order (brute force on a permutation)
            for perm in itertools.permutations(c):
                bt = brute.table(geno, pheno, perm)
                assert O.mi(bt[0], bt[1], m) == pytest.approx(v, rel=1e-12, abs=1e-15)
            # adding a SNP never lowers MI
            if k > 1:
                for d in range(k):
                    sub = tuple(s for i, s in enumerate(c) if i != d)
                    assert v >= mi_of[sub] - 1e-12


# ----------------------------------------------------------------------------
# exhaustive search with top-N retention
# ----------------------------------------------------------------------------

def _all_sorted(geno, pheno, k):
    m = geno.shape[1]
    rows = []
    for c in brute.all_combinations(geno.shape[0], k):
        t = brute.table(geno, pheno, c)
        rows.append((-O.mi(t[0], t[1], m), c))
    rows.sort()
    return rows


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("threads", [1, 3])
def test_search_matches_full_sort(oracle_lib, k, threads):
    n, m = 10, 67
    geno, pheno = _rand(n, m, seed=40 + k)
    geno[7] = geno[2]           # duplicated SNPs create exact ties
    geno[9] = geno[4]
    full = _all_sorted(geno, pheno, k)
    for top_n in (1, 5, len(full), len(full) + 3):
        combs, mis, counts = O.search(geno, pheno, k, top_n, threads=threads)
        want = full[:top_n]
        assert len(combs) == len(want)
        assert [tuple(c) for c in combs.tolist()] == [c for _, c in want]
        assert mis.tolist() == [-v for v, _ in want]
        for c, t in zip(combs, counts):
            assert t.tolist() == brute.table(geno, pheno, tuple(c)).tolist()


def test_search_rank_ranges(oracle_lib):
    n, m, k = 11, 50, 3
    geno, pheno = _rand(n, m, seed=77)
    allc = brute.all_combinations(n, k)
    for (r0, r1) in [(0, 1), (5, 40), (100, 165), (160, 10 ** 6)]:
        sub = allc[r0:r1]
        rows = []
        for c in sub:
            t = brute.table(geno, pheno, c)
            rows.append((-O.mi(t[0], t[1], m), c))
        rows.sort()
        combs, mis, _ = O.search(geno, pheno, k, 7, rank_begin=r0, rank_end=r1, threads=2)
        assert [tuple(c) for c in combs.tolist()] == [c for _, c in rows[:7]]


def test_search_recovers_planted_pair(oracle_lib):
    from paper_2201_02460_gb300 import synth
    ds, k, top_n = synth.make_workload("order2_200snp_1600")
    combs, mis, counts = O.search(ds.geno, ds.pheno, k, top_n)
    assert tuple(combs[0]) == ds.planted
    assert mis[0] > 5 * mis[1]
    # no marginal effect of the planted SNPs (parity penetrance at MAF 0.5)
    c1, m1_, _ = O.search(ds.geno, ds.pheno, 1, 200)
    ranks = {int(c[0]): i for i, c in enumerate(c1)}
    assert all(ranks[s] > 10 for s in ds.planted)


def test_search_all_zero_scores_lexicographic(oracle_lib):
    # a single phenotype class makes every MI exactly zero: lex order decides
    geno, pheno = _rand(8, 30, seed=5, m1=0)
    combs, mis, _ = O.search(geno, pheno, 3, 10)
    assert (mis == 0.0).all()
    assert [tuple(c) for c in combs.tolist()] == brute.all_combinations(8, 3)[:10]
