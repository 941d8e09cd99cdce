"""Comparison helpers shared by the GPU parity tests."""
from __future__ import annotations

import numpy as np

# |MI_gpu64 - MI_oracle| bound in nats: both are double precision; the oracle
# evaluates Eq. 1 as a difference of entropies (magnitudes up to ln(2 * 3^k)
# ~ 6.2 for k = 5, a few hundred terms), which loses at most ~1e-13.
F64_ATOL = 1e-12
# single-precision screening score: relative bound asked of the FP32 path
F32_RTOL = 1e-6


def check_topn(g_combs, g_mi, o_combs, o_mi, atol=F64_ATOL):
    """GPU top-N against the oracle's: identical scores (within atol), and
    identical combinations except inside groups of equal scores, whose order
    is not unique."""
    g_combs = [tuple(int(x) for x in c) for c in g_combs]
    o_combs = [tuple(int(x) for x in c) for c in o_combs]
    assert len(g_combs) == len(o_combs), (len(g_combs), len(o_combs))
    n = len(o_combs)
    if n == 0:
        return
    np.testing.assert_allclose(np.asarray(g_mi), np.asarray(o_mi), rtol=0, atol=atol)
    o_mi = np.asarray(o_mi)
    for i in range(n):
        if g_combs[i] != o_combs[i]:
            tied = [j for j in range(n) if abs(o_mi[j] - o_mi[i]) <= atol and j != i]
            assert tied or i == n - 1, f"rank {i}: gpu {g_combs[i]} vs oracle {o_combs[i]} (no tie)"
    cut = o_mi[-1] + atol
    gs = {c for c, v in zip(g_combs, o_mi) if v > cut}
    os_ = {c for c, v in zip(o_combs, o_mi) if v > cut}
    assert gs == os_
    assert len(set(g_combs)) == n, "duplicate combinations"


def random_data(n, m, seed, m1=None, p_levels=(0.2, 0.5)):
    rng = np.random.default_rng(seed)
    maf = rng.uniform(*p_levels, size=n)
    u = rng.random((n, m))
    q = 1 - maf[:, None]
    geno = ((u >= q * q).astype(np.uint8) + (u >= q * q + 2 * maf[:, None] * q).astype(np.uint8))
    if m1 is None:
        pheno = rng.integers(0, 2, size=m, dtype=np.uint8)
    else:
        pheno = np.zeros(m, np.uint8)
        pheno[rng.choice(m, size=m1, replace=False)] = 1
    return geno.astype(np.uint8), pheno
