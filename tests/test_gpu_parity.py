"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Counts and top-N combinations must match bit for bit; double-precision
scores within F64_ATOL; the single-precision screening score within 1e-6
relative of the oracle's double-precision MI.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import brute
from oracle import oracle as O
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


@pytest.fixture(params=["auto", "separate"])
def tc_variant(request, ctx):
    """Runs a tensor-path test with the combined-class variant where it
    applies ("auto") and with separate class accumulators; restores auto."""
    ctx.set_tc_variant(request.param)
    yield request.param
    ctx.set_tc_variant("auto")


def comb_shift(m1, m0, k):
    """The combined-class variant's class shift (0: not applicable), the
    rule the library documents for EPI_TC_AUTO."""
    if k != 3:
        return 0
    p = 1
    while p < 15 and (1 << p) <= m0:
        p += 1
    if p > 14 or m1 * (1 << p) + m0 >= (1 << 23):
        return 0
    return p


def _search_both(epi, ctx, geno, pheno, k, top_n, path="popc", rank_range=None):
    ds = epi.Dataset(ctx, geno, pheno)
    r = epi.search(ds, k, top_n, path=path, rank_range=rank_range)
    if rank_range is None:
        oc, om, ot = O.search(geno, pheno, k, top_n)
    else:
        oc, om, ot = O.search(geno, pheno, k, top_n, rank_begin=rank_range[0], rank_end=rank_range[1])
    return ds, r, oc, om, ot


def _check_result(r, geno, pheno, oc, om):
    check_topn(r.combs, r.mi, oc, om)
    # every returned table is the oracle's table of that combination
    if len(r):
        t = O.tables(geno, pheno, r.combs.astype(np.int32))
        assert (t == r.counts).all()
        m = geno.shape[1]
        want = np.array([O.mi(x[0], x[1], m) for x in t])
        np.testing.assert_allclose(r.mi, want, rtol=0, atol=F64_ATOL)
        err = np.abs(r.mi_f32.astype(np.float64) - want)
        assert (err <= F32_RTOL * want + 1e-12).all(), err.max()
        # ranks are lexicographic ranks
        for c, rk in zip(r.combs[:20], r.rank[:20]):
            assert O.rank(geno.shape[0], r.order, c) == int(rk)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("m", [37, 128, 129, 300])
def test_tables_match_oracle(epi, ctx, k, m):
    geno, pheno = random_data(11, m, seed=k * 1000 + m)
    ds = epi.Dataset(ctx, geno, pheno)
    combs = np.array(brute.all_combinations(11, k), dtype=np.uint32)
    got = epi.tables(ds, combs)
    want = O.tables(geno, pheno, combs.astype(np.int32))
    assert (got == want).all()


def test_tables_high_order(epi, ctx):
    geno, pheno = random_data(10, 90, seed=8)
    ds = epi.Dataset(ctx, geno, pheno)
    for k in (6, 7, 8):
        combs = np.array(brute.all_combinations(10, k)[:40], dtype=np.uint32)
        assert (epi.tables(ds, combs) == O.tables(geno, pheno, combs.astype(np.int32))).all()


@pytest.mark.parametrize("k,n,m,top_n", [
    (1, 30, 200, 10), (2, 40, 257, 25), (3, 30, 700, 50), (4, 22, 1100, 40), (5, 16, 450, 30),
    (2, 12, 64, 66), (3, 9, 33, 200),
])
def test_search_small(epi, ctx, k, n, m, top_n):
    geno, pheno = random_data(n, m, seed=7 * k + n)
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, top_n)
    _check_result(r, geno, pheno, oc, om)


# Orders 6-8 (popcount path; the tensor path stops at 5).  Single searches
# stage (k-2)-prefix tables in shared memory with a single-count table per
# prefix and count last pairs (whole rounds of one pair per warp, then the
# last pairs' rows split over warps);
# batched launches and the thresholded output keep (k-1)-prefix tables
# (test_batched_high_orders, test_search_threshold_matches_oracle).
@pytest.mark.parametrize("k,n,m,m1,top_n", [
    (6, 14, 300, None, 40), (6, 12, 129, 40, 20), (7, 13, 700, None, 30), (7, 11, 3000, 1500, 20),
    (8, 12, 200, None, 25), (8, 11, 1000, 500, 15),
])
def test_search_high_orders(epi, ctx, k, n, m, m1, top_n):
    geno, pheno = random_data(n, m, seed=13 * k + n, m1=m1)
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, top_n)
    _check_result(r, geno, pheno, oc, om)


@pytest.mark.parametrize("k,m,m1", [(6, 700, None), (7, 3000, 1500), (8, 200, None)])
def test_search_range_high_orders(epi, ctx, k, m, m1):
    n = {6: 16, 7: 14, 8: 13}[k]
    geno, pheno = random_data(n, m, seed=31 + k, m1=m1)
    total = O.binom(n, k)
    for r0, r1 in [(0, 1), (17, 1000), (total - 100, total + 10)]:
        ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, 20, rank_range=(r0, r1))
        _check_result(r, geno, pheno, oc, om)
        assert all(r0 <= int(x) < r1 for x in r.rank)


def test_workload_order8_table2_ranges(epi, ctx):
    """The order-8 row of Table 2 (23 SNPs x 2048 samples) at full size, on
    rank ranges the oracle covers quickly: the first, a middle and the last
    3000 combinations."""
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload("order8_23snp_2048")
    total = O.binom(d.n_snps, k)
    for r0 in (0, total // 2, total - 3000):
        ds, r, oc, om, _ = _search_both(epi, ctx, d.geno, d.pheno, k, 25, rank_range=(r0, r0 + 3000))
        _check_result(r, d.geno, d.pheno, oc, om)


@pytest.mark.parametrize("k,n,m,chunk", [(2, 40, 300, 0), (3, 16, 257, 100), (5, 12, 400, 0), (7, 11, 300, 77)])
def test_search_threshold_matches_oracle(epi, ctx, k, n, m, chunk):
    """Thresholded output: every combination with MI >= threshold, best
    first, with its table; a capacity below the count keeps the best; a
    threshold of 0 takes every combination and one above the maximum none.
    Small chunks make several scoring passes."""
    geno, pheno = random_data(n, m, seed=5 * k + n)
    ds = epi.Dataset(ctx, geno, pheno)
    total = O.binom(n, k)
    oc, om, _ = O.search(geno, pheno, k, total)
    # a threshold between two distinct values, about 40 combinations in
    i = next(i for i in range(min(40, total - 1), total) if om[i - 1] - om[i] > 1e-9 * max(om[i], 1e-12))
    thr = 0.5 * (om[i - 1] + om[i])
    r, nf = epi.search_threshold(ds, k, thr, capacity=total, chunk=chunk)
    assert nf == i and len(r) == i
    check_topn(r.combs, r.mi, oc[:i], om[:i])
    assert (r.counts == O.tables(geno, pheno, r.combs.astype(np.int32))).all()
    r2, nf2 = epi.search_threshold(ds, k, thr, capacity=5, chunk=chunk)
    assert nf2 == i and len(r2) == 5
    check_topn(r2.combs, r2.mi, oc[:5], om[:5])
    _, nf3 = epi.search_threshold(ds, k, 0.0, capacity=0, chunk=chunk, with_counts=False)
    assert nf3 == total
    _, nf4 = epi.search_threshold(ds, k, om[0] * 1.001 + 1e-9, capacity=10, chunk=chunk)
    assert nf4 == 0


def test_batched_high_orders(epi, ctx):
    """Orders 6-8 in one batched launch per order (prefix tables in shared
    memory: 729 rows x 12 words at order 7, 2187 x 8 at order 8) match the
    single searches (global tables at orders 7-8) and the oracle."""
    sets = [random_data(n, m, seed=70 + i) for i, (n, m) in enumerate([(12, 300), (11, 350), (11, 200), (12, 180)])]
    orders, tops = [6, 7, 8, 7], [15, 12, 10, 9]
    dss = [epi.Dataset(ctx, g, p) for g, p in sets]
    res = epi.search_batched(ctx, dss, orders, tops, path="popc")
    for (g, p), ds, k, t, r in zip(sets, dss, orders, tops, res):
        single = epi.search(ds, k, t, path="popc")
        oc, om, _ = O.search(g, p, k, t)
        _check_result(r, g, p, oc, om)
        assert (r.combs == single.combs).all() and np.array_equal(r.mi, single.mi)


@pytest.mark.parametrize("path,k,world", [("popc", 3, 3), ("tc", 3, 3), ("tc", 4, 5), ("tc", 2, 4)])
def test_sharded_ranges_merge_to_the_full_search(epi, ctx, path, k, world, tc_variant):
    """The sharding hook on the GPU: every range search of a rank split
    against the oracle's search of the same range, and the ranges' records,
    merged by (MI desc, rank asc), against the oracle's whole top-N."""
    from paper_2201_02460_gb300 import shard
    n = {2: 200, 3: 60, 4: 30}[k]
    geno, pheno = random_data(n, 700, seed=21 + k)
    ds = epi.Dataset(ctx, geno, pheno)
    t = 40
    total = O.binom(n, k)
    parts = []
    for b, e in shard.rank_ranges(total, world):
        r = epi.search(ds, k, t, path=path, rank_range=(b, e))
        oc, om, _ = O.search(geno, pheno, k, t, rank_begin=b, rank_end=e)
        _check_result(r, geno, pheno, oc, om)
        assert all(b <= int(x) < e for x in r.rank)
        parts.append(r.records)
    got = shard.merge_topn(parts, t)
    oc, om, _ = O.search(geno, pheno, k, t)
    check_topn(got["snp"][:, :k], got["mi"], oc, om)


def test_search_with_exact_ties(epi, ctx):
    geno, pheno = random_data(24, 301, seed=99)
    geno[10] = geno[3]
    geno[17] = geno[5]
    geno[20] = geno[3]
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, 3, 60)
    _check_result(r, geno, pheno, oc, om)


@pytest.mark.parametrize("m1", [0, 1, 299])
def test_search_single_or_nearly_single_class(epi, ctx, m1):
    geno, pheno = random_data(15, 300, seed=5, m1=m1)
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, 3, 40)
    _check_result(r, geno, pheno, oc, om)


@pytest.mark.parametrize("path", ["popc", "tc"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_search_range(epi, ctx, k, path, tc_variant):
    n = {2: 300, 3: 80, 4: 40, 5: 24}[k]
    geno, pheno = random_data(n, 513, seed=11 + k)
    total = O.binom(n, k)
    for r0, r1 in [(0, 1), (17, 5000), (total // 3, total // 3 + 77777), (total - 999, total + 10),
                   (total // 2, total // 2 + 1)]:
        ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, 30, path=path, rank_range=(r0, r1))
        _check_result(r, geno, pheno, oc, om)
        assert all(r0 <= int(x) < r1 for x in r.rank)


def test_workload_order2_full(epi, ctx):
    from paper_2201_02460_gb300 import synth
    ds_, k, top_n = synth.make_workload("order2_200snp_1600")
    for N in (top_n, 1000):
        ds, r, oc, om, _ = _search_both(epi, ctx, ds_.geno, ds_.pheno, k, N)
        _check_result(r, ds_.geno, ds_.pheno, oc, om)
    assert tuple(r.combs[0]) == ds_.planted


def test_workload_order3_reduced(epi, ctx):
    """The order-3 workload with 4000 samples at 260 SNPs (2.9M combinations,
    several tiles per CTA and ragged sub-tiles): full oracle parity."""
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload("order3_2000snp_4000", n_snps=260)
    ds, r, oc, om, _ = _search_both(epi, ctx, d.geno, d.pheno, k, top_n)
    _check_result(r, d.geno, d.pheno, oc, om)


def test_workload_order4_reduced(epi, ctx):
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload("order4_500snp_8192", n_snps=48)
    ds, r, oc, om, _ = _search_both(epi, ctx, d.geno, d.pheno, k, top_n)
    _check_result(r, d.geno, d.pheno, oc, om)


def test_device_inputs_match_host_inputs(epi, ctx):
    import torch
    geno, pheno = random_data(40, 999, seed=3)
    a = epi.search(epi.Dataset(ctx, geno, pheno), 3, 50)
    b = epi.search(epi.Dataset(ctx, torch.from_numpy(geno).cuda(), torch.from_numpy(pheno).cuda()), 3, 50)
    assert (a.records == b.records).all()


def test_search_async_matches_sync(epi, ctx):
    import torch
    geno, pheno = random_data(50, 800, seed=4)
    ds = epi.Dataset(ctx, geno, pheno)
    a = epi.search(ds, 3, 64)
    out = torch.zeros(64 * 56, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros((64, 2, 27), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    epi.search_async(ds, 3, 64, out, cnt, n_out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(n_out.item()) == 64
    recs = np.frombuffer(out.cpu().numpy().tobytes(), dtype=epi.RESULT_DTYPE)
    assert (recs == a.records).all()
    assert (cnt.cpu().numpy().astype(np.uint32) == a.counts).all()


def test_invalid_inputs(epi, ctx):
    geno, pheno = random_data(8, 50, seed=1)
    bad = geno.copy()
    bad[3, 7] = 3
    with pytest.raises(epi.EpiError) as e:
        epi.Dataset(ctx, bad, pheno)
    assert e.value.status == epi.EPI_EINVAL
    badp = pheno.copy()
    badp[0] = 2
    with pytest.raises(epi.EpiError):
        epi.Dataset(ctx, geno, badp)
    ds = epi.Dataset(ctx, geno, pheno)
    for k, n in [(0, 5), (9, 5), (3, 0), (3, 5000)]:
        with pytest.raises(epi.EpiError) as e:
            epi.search(ds, k, n)
        assert e.value.status == epi.EPI_EINVAL
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 6, 5, path="tc")
    assert e.value.status == epi.EPI_EUNSUPPORTED
    with pytest.raises(epi.EpiError):
        epi.tables(ds, np.array([[3, 3]], dtype=np.uint32))
    with pytest.raises(epi.EpiError):
        epi.tables(ds, np.array([[1, 8]], dtype=np.uint32))


def test_score_tables_fp32_accuracy(epi, ctx):
    """The single-precision screening score on random tables of every order:
    within 1e-6 relative of the oracle's double-precision MI."""
    rng = np.random.default_rng(12)
    geno, pheno = random_data(6, 4096, seed=2, m1=2000)
    ds = epi.Dataset(ctx, geno, pheno)
    for k in (1, 2, 3, 4, 5):
        cells = 3 ** k
        tabs = []
        for _ in range(200):
            a = rng.multinomial(2000, rng.dirichlet(np.ones(cells)))
            b = rng.multinomial(2096, rng.dirichlet(np.ones(cells)))
            tabs.append([a, b])
        tabs = np.array(tabs, dtype=np.uint32)
        f32, f64 = epi.score_tables(ds, k, tabs)
        want = np.array([O.mi(t[0], t[1], 4096) for t in tabs])
        np.testing.assert_allclose(f64, want, rtol=0, atol=F64_ATOL)
        assert (np.abs(f32 - want) <= F32_RTOL * want + 1e-12).all()


# ---------------------------------------------------------------------------
# tensor-core counting path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k,n,m,m1", [(2, 50, 300, None), (3, 24, 700, None), (3, 40, 129, None),
                                      (4, 14, 1000, None), (4, 12, 257, None), (3, 70, 2000, None),
                                      (2, 150, 64, None), (5, 12, 700, None), (5, 16, 129, None), (5, 30, 1000, None),
                                      (3, 100, 4000, None), (3, 150, 700, None), (3, 20, 6000, 1000), (3, 18, 6000, 1020),
                                      (3, 16, 6000, 1100)])
def test_tc_counts_bit_exact(epi, ctx, k, n, m, m1, tc_variant):
    """Every combination's table from the tensor-core kernel equals the
    popcount table kernel's and the oracle's, bit for bit.  Two order-3
    cases sit at the combined-class variant's limit: m1 2^13 + m0 just below
    2^23 (1000 cases over 5000 controls) and just above it (1100 cases: the
    separate-class variant runs)."""
    geno, pheno = random_data(n, m, seed=300 * k + n + m, m1=m1)
    if m1 is not None and tc_variant == "auto" and k == 3:
        assert (comb_shift(m1, m - m1, k) != 0) == (m1 <= 1020)
    ds = epi.Dataset(ctx, geno, pheno)
    got = epi.debug_counts(ds, k)
    combs = np.array(brute.all_combinations(n, k), dtype=np.uint32)
    want = epi.tables(ds, combs)
    assert (want == O.tables(geno, pheno, combs.astype(np.int32))).all()
    bad = np.nonzero((got != want).any(axis=(1, 2)))[0]
    assert len(bad) == 0, f"{len(bad)} tables differ, first rank {bad[:5]}"


@pytest.mark.parametrize("k,n,m,top_n", [(2, 60, 257, 25), (3, 30, 700, 50), (3, 90, 1500, 100),
                                         (4, 22, 1100, 40), (4, 30, 513, 64), (5, 18, 900, 40),
                                         (5, 26, 400, 100)])
def test_tc_search_small(epi, ctx, k, n, m, top_n, tc_variant):
    geno, pheno = random_data(n, m, seed=11 * k + n)
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, top_n, path="tc")
    _check_result(r, geno, pheno, oc, om)


def test_tc_matches_popc(epi, ctx, tc_variant):
    geno, pheno = random_data(120, 2000, seed=77)
    geno[50] = geno[7]
    ds = epi.Dataset(ctx, geno, pheno)
    a = epi.search(ds, 3, 200, path="popc")
    b = epi.search(ds, 3, 200, path="tc")
    assert (a.combs == b.combs).all()
    assert (a.mi == b.mi).all()
    assert (a.counts == b.counts).all()
    np.testing.assert_allclose(a.mi_f32, b.mi_f32, rtol=2e-6)


def test_tc_matches_popc_order5(epi, ctx):
    # order 5: one prefix per tile, a combination summed across three warps
    geno, pheno = random_data(90, 2000, seed=78)
    geno[40] = geno[3]
    ds = epi.Dataset(ctx, geno, pheno)
    a = epi.search(ds, 5, 150, path="popc")
    b = epi.search(ds, 5, 150, path="tc")
    assert (a.combs == b.combs).all()
    assert (a.mi == b.mi).all()
    assert (a.counts == b.counts).all()
    np.testing.assert_allclose(a.mi_f32, b.mi_f32, rtol=2e-6)


def test_tc_workload_order3_reduced(epi, ctx):
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload("order3_2000snp_4000", n_snps=260)
    ds, r, oc, om, _ = _search_both(epi, ctx, d.geno, d.pheno, k, top_n, path="tc")
    _check_result(r, d.geno, d.pheno, oc, om)


def test_tc_workload_order4_reduced(epi, ctx):
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload("order4_500snp_8192", n_snps=48)
    ds, r, oc, om, _ = _search_both(epi, ctx, d.geno, d.pheno, k, top_n, path="tc")
    _check_result(r, d.geno, d.pheno, oc, om)


def test_tc_unsupported_cases(epi, ctx):
    geno, pheno = random_data(20, 100, seed=1, m1=0)
    ds = epi.Dataset(ctx, geno, pheno)
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 3, 10, path="tc")
    assert e.value.status == epi.EPI_EUNSUPPORTED
    geno, pheno = random_data(20, 100, seed=1)
    ds = epi.Dataset(ctx, geno, pheno)
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 6, 10, path="tc")
    assert e.value.status == epi.EPI_EUNSUPPORTED
    # a short range: auto takes the popcount path, the tensor path still
    # answers when asked for
    r = epi.search(ds, 3, 10, path="auto", rank_range=(0, 100))
    assert len(r) == 10
    t = epi.search(ds, 3, 10, path="tc", rank_range=(0, 100))
    assert (t.combs == r.combs).all()


def test_profile_trace_survives_scratch_growth(epi, ctx):
    """The wait trace of a tensor-core search stays readable after a later
    search grew the context's scratch memory."""
    geno, pheno = random_data(120, 1500, seed=8)
    ds = epi.Dataset(ctx, geno, pheno)
    ctx.profile_begin()
    epi.search(ds, 3, 50, path="tc")
    epi.search(ds, 3, 1000, path="popc")      # larger candidate lists
    w = ctx.profile_waits()
    ms, n = ctx.profile_end()
    assert n == 2 and ms > 0
    assert w["mma_loop"] > 0


# ---------------------------------------------------------------------------
# batched searches
# ---------------------------------------------------------------------------

def _batch_case(seed):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(10):
        k = int(rng.integers(1, 6))
        n = int(rng.integers(k + 2, {1: 300, 2: 120, 3: 60, 4: 30, 5: 18}[k]))
        m = int(rng.integers(40, 2500))
        m1 = int(rng.integers(1, m)) if i % 4 else int(rng.integers(0, 2)) * m
        specs.append((k, n, m, m1, int(rng.integers(1, 80))))
    return specs


@pytest.mark.parametrize("path", ["auto", "popc"])
def test_batched_matches_single(epi, ctx, path):
    specs = _batch_case(5)
    data = [random_data(n, m, seed=100 + i, m1=m1) for i, (k, n, m, m1, t) in enumerate(specs)]
    dss = [epi.Dataset(ctx, g, p) for g, p in data]
    orders = [s[0] for s in specs]
    tops = [s[4] for s in specs]
    for rep in range(2):                       # capture, then replay
        res = epi.search_batched(ctx, dss, orders, tops, path=path)
        for ds, k, t, r in zip(dss, orders, tops, res):
            one = epi.search(ds, k, t, path=path)
            assert (r.records == one.records).all()
            assert (r.counts == one.counts).all()


def test_batched_against_oracle_and_new_graph(epi, ctx):
    specs = [(3, 40, 900, 400, 30), (2, 90, 1300, 650, 25), (4, 20, 700, 300, 20), (3, 50, 2100, 1000, 40)]
    data = [random_data(n, m, seed=7 + i, m1=m1) for i, (k, n, m, m1, t) in enumerate(specs)]
    dss = [epi.Dataset(ctx, g, p) for g, p in data]
    res = epi.search_batched(ctx, dss, [s[0] for s in specs], [s[4] for s in specs])
    for (g, p), (k, n, m, m1, t), r in zip(data, specs, res):
        oc, om, ot = O.search(g, p, k, t)
        _check_result(r, g, p, oc, om)
    # different top_n: a new graph
    res2 = epi.search_batched(ctx, dss, [s[0] for s in specs], [5, 6, 7, 8])
    for r, r_old in zip(res2, res):
        assert (r.records == r_old.records[: len(r)]).all()


def test_autotune_choices_and_results(epi, ctx, tmp_path):
    for k, n, m in [(3, 70, 1500), (4, 26, 2000)]:
        geno, pheno = random_data(n, m, seed=21 + k)
        ds = epi.Dataset(ctx, geno, pheno)
        before = epi.search(ds, k, 40)
        t = epi.autotune(ds, k)
        assert t["row_group"] in ((9,) if k == 3 else (9, 27))
        assert t["tile"] in (128, 256, 512) and t["slots"] in (1, 2, 4, 8) and t["path"] in ("popc", "tc")
        after = epi.search(ds, k, 40)
        assert (after.records["snp"] == before.records["snp"]).all() and (after.mi == before.mi).all()
        forced = epi.search(ds, k, 40, path="popc")
        assert (forced.combs == before.combs).all()
    f = tmp_path / "tune.txt"
    epi.tune_save(ctx, str(f))
    lines = [x for x in f.read_text().splitlines() if not x.startswith("#")]
    assert len(lines) >= 2
    ctx2 = epi.Context(0)
    epi.tune_load(ctx2, str(f))
    epi.tune_save(ctx2, str(tmp_path / "again.txt"))
    assert (tmp_path / "again.txt").read_text() == f.read_text()


def test_batched_config4_shapes(epi, ctx):
    """The 64 seeded dataset shapes of the batched configuration (orders
    2-4, 1000-16000 samples, case fraction 0.3-0.7) at reduced SNP counts:
    the batch equals the per-dataset searches, and a sample equals the
    oracle."""
    from paper_2201_02460_gb300 import synth
    specs = synth.batch_specs()
    dss, orders, tops, raw = [], [], [], []
    for sp in specs:
        n = max(sp["order"] + 2, sp["n_snps"] // {2: 10, 3: 25, 4: 60}[sp["order"]])
        d = synth.make_dataset(n, sp["n_cases"], sp["n_controls"], seed=sp["seed"], maf_lo=sp["maf_lo"])
        dss.append(epi.Dataset(ctx, d.geno, d.pheno))
        orders.append(sp["order"])
        tops.append(sp["top_n"])
        raw.append(d)
    res = epi.search_batched(ctx, dss, orders, tops)
    for i, (ds, k, t, r) in enumerate(zip(dss, orders, tops, res)):
        one = epi.search(ds, k, t)
        assert (r.records == one.records).all(), i
        if i % 8 == 0:
            oc, om, _ = O.search(raw[i].geno, raw[i].pheno, k, t)
            _check_result(r, raw[i].geno, raw[i].pheno, oc, om)


def test_tc_rate_probe(epi, ctx):
    """The tensor-pipe rate probe returns a consistent measurement: the rate
    from event time and the per-SM cycle count agree with the SM clock it
    reports, and the count per clock lies below the nominal dense FP8 bound
    (4.5 PFLOP/s at about 1.9 GHz over 152 SMs: under 8 Ki multiply-adds per
    SM clock, with 20 % headroom for clock reporting)."""
    for shape in (0, 1):
        r = ctx.tc_rate(1 << 14, shape=shape)
        assert r["ms"] > 0 and r["tflops"] > 0
        assert 0 < r["mac_per_clk_sm"] <= 1.2 * 8192
        implied = r["tflops"] * 1e12 / (2 * r["mac_per_clk_sm"] * 152) / 1e6
        assert 0.8 * r["sm_mhz"] <= implied <= 1.25 * r["sm_mhz"]
    with pytest.raises(epi.EpiError):
        ctx.tc_rate(1 << 14, shape=2)


@pytest.mark.parametrize("k,n,m,m1", [(2, 40, 300, 140), (3, 20, 777, 400), (4, 13, 1000, 313), (3, 18, 4100, 2049),
                                      (2, 30, 65, 1)])
def test_count_variants_bit_exact(epi, ctx, k, n, m, m1):
    """The three last-level counting instructions (POPC, byte lookup table,
    binary MMA AND+POPC) give every table of the oracle, and the same
    checksum."""
    geno, pheno = random_data(n, m, seed=500 + 7 * k + m, m1=m1)
    ds = epi.Dataset(ctx, geno, pheno)
    combs = np.array(brute.all_combinations(n, k), dtype=np.int32)
    want = O.tables(geno, pheno, combs)
    cells = 3 ** k
    weights = 1 + np.arange(cells, dtype=np.uint64)[None, None, :] + np.array([0, cells], dtype=np.uint64)[None, :, None]
    want_sum = int((want.astype(np.uint64) * weights).sum())
    for v in ("popc", "lut", "mma_b1"):
        r = epi.count_variant(ds, k, v, with_tables=True)
        bad = np.nonzero((r["tables"] != want).any(axis=(1, 2)))[0]
        assert len(bad) == 0, (v, len(bad), bad[:5])
        assert r["checksum"] == want_sum % (1 << 64), v


@pytest.mark.parametrize("k,n", [(3, 60), (4, 26)])
def test_tc_large_top_n(epi, ctx, k, n, tc_variant):
    """top_n = 1024: the candidate pool (1088) no longer fits beside the
    operand rings, so the tensor kernel keeps its candidate lists in global
    memory; the result is still the oracle's."""
    geno, pheno = random_data(n, 900, seed=40 + k)
    ds, r, oc, om, _ = _search_both(epi, ctx, geno, pheno, k, 1024, path="tc")
    _check_result(r, geno, pheno, oc, om)
