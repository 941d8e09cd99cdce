"""Host-side arithmetic of bench.py (no GPU): the work counts behind the
roofline fractions, checked against enumeration on small cases."""
from __future__ import annotations

import itertools
import math
import types

import bench


def _ds(n, m, m1):
    return types.SimpleNamespace(n_snps=n, n_samples=m, n_cases=m1)


def _words(d):
    return 4 * (-(-d.n_cases // 128) + -(-(d.n_samples - d.n_cases) // 128))


def test_popc_executed_ops_matches_enumeration():
    """Orders 6-8: per (k-2)-prefix with L >= 2 following SNPs, 3^(k-2) rows x
    words x (4 joint counts per pair + 2 single counts per following SNP + 1
    row total); below order 6, two genotype rows per (k-1)-prefix row."""
    for n, k in [(9, 6), (10, 7), (11, 8), (12, 6)]:
        d = _ds(n, 700, 300)
        W = _words(d)
        want = 0
        for pre in itertools.combinations(range(n), k - 2):
            L = n - 1 - pre[-1]
            if L >= 2:
                want += 3 ** (k - 2) * W * (4 * math.comb(L, 2) + 2 * L + 1)
        assert bench.popc_executed_ops(d, k, W) == want
        # every combination belongs to exactly one prefix's pairs
        assert sum(math.comb(n - 1 - p[-1], 2) for p in itertools.combinations(range(n), k - 2)) == math.comb(n, k)
    for n, k in [(20, 3), (12, 5)]:
        d = _ds(n, 700, 300)
        W = _words(d)
        assert bench.popc_executed_ops(d, k, W) == math.comb(n, k) * 2 * 3 ** (k - 1) * W


def test_popc_roofline_fractions():
    """Paper work counts 3^k cells x words per combination; the executed
    fraction divides the same time into the kernel's own POPC count."""
    d = _ds(23, 2048, 1024)
    ms = 34.1
    r = bench.roofline("popc", d, 8, ms, {"bf16": 1.0, "source": "test"})
    W = _words(d)
    peak = 152 * 16 * 2070e6
    assert math.isclose(r["frac"], math.comb(23, 8) * 3 ** 8 * W / (ms / 1e3) / peak, rel_tol=1e-12)
    assert math.isclose(r["executed_frac"], bench.popc_executed_ops(d, 8, W) / (ms / 1e3) / peak, rel_tol=1e-12)
    assert r["kernel"] == "popc_pair_kernel" and r["executed_frac"] < r["frac"]
    r3 = bench.roofline("popc", _ds(2000, 4000, 2000), 3, 968.0, {"bf16": 1.0, "source": "test"})
    assert r3["kernel"] == "popc_search_kernel"
    assert math.isclose(r3["executed_frac"] / r3["frac"], 2.0 / 3.0, rel_tol=1e-12)


def test_comb_shift_rule():
    """The combined-class variant's shift p: the least p with 2^p > m0, used
    only at order 3 while p <= 14 and m1 * 2^p + m0 < 2^23."""
    assert bench.comb_shift(_ds(2000, 4000, 2000), 3) == 11        # 2^11 = 2048 > 2000
    assert bench.comb_shift(_ds(2000, 4000, 2000), 4) == 0
    assert bench.comb_shift(_ds(500, 8192, 4096), 3) == 0           # 4096 * 2^13 + 4096 >= 2^23
    assert bench.comb_shift(_ds(500, 5000, 1000), 3) == 12          # 2^12 > 4000; 1000 * 4096 + 4000 < 2^23
    assert bench.comb_shift(_ds(500, 1025, 1024), 3) == 1           # one control
    for m, m1 in [(4000, 2000), (5000, 1000), (1600, 800), (16000, 5000), (9000, 1020)]:
        p = bench.comb_shift(_ds(100, m, m1), 3)
        m0 = m - m1
        if p:
            assert (1 << p) > m0 >= (1 << (p - 1)) or (p == 1 and m0 < 2)
            assert m1 * (1 << p) + m0 < (1 << 23) and p <= 14
