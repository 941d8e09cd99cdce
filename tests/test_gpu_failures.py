"""Failure paths of the search, driven without faulting the GPU.

* Exact ties at the pool boundary: copies of one SNP give combinations with
  identical tables, hence identical MI in both precisions.  The exact top-N
  (MI desc, rank asc) cannot be proven from a pool that holds only some of the
  tied combinations, so the search widens its candidate pool (4x per retry)
  until every tie fits, and returns EPI_EOVERFLOW when even the largest pool
  (4096) cannot hold them.
* A bounded device wait that gives up: the context's wait limit is set to a
  microsecond, so the tensor-core kernel's first pipeline wait (for an
  accumulator that takes several microseconds to fill) runs out; every role
  drains its own work and the call returns EPI_ETIMEOUT.  With the limit back
  at its default the same context searches correctly.
* A device allocation that fails: the context's allocation wrapper is told to
  fail once; the call returns EPI_ENOMEM and the context keeps working.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.helpers import check_topn, random_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_02460_gb300 import epi as E
    E.load()
    return E


def _copies(n, m, seed):
    geno, pheno = random_data(n, m, seed=seed)
    geno[:] = geno[0]
    return geno, pheno


@pytest.mark.parametrize("path", ["popc", "tc"])
def test_exact_ties_widen_the_pool(epi, path):
    ctx = epi.Context(0)
    # C(60, 2) = 1770 combinations with one identical table: more than the
    # first pools (128, 512) hold, fewer than 2048
    geno, pheno = _copies(60, 700, seed=3)
    ds = epi.Dataset(ctx, geno, pheno)
    plain_geno, _ = random_data(60, 700, seed=4)
    plain = epi.Dataset(ctx, plain_geno, pheno)
    epi.search(plain, 2, 10, path=path)          # first search: builds the operand tables
    l0 = ctx.kernel_launches()
    epi.search(plain, 2, 10, path=path)
    one_pass = ctx.kernel_launches() - l0
    l0 = ctx.kernel_launches()
    r = epi.search(ds, 2, 10, path=path)
    passes = (ctx.kernel_launches() - l0) / one_pass
    assert passes >= 3, passes           # pools 128 and 512 could not prove it
    oc, om, ot = O.search(geno, pheno, 2, 10)
    check_topn(r.combs, r.mi, oc, om)
    # all tied: the lexicographically first pairs, in rank order
    assert [tuple(c) for c in r.combs.tolist()] == [(0, j) for j in range(1, 11)]
    assert (r.counts == ot).all()


@pytest.mark.parametrize("path", ["popc", "tc"])
def test_too_many_exact_ties_report_eoverflow(epi, path):
    ctx = epi.Context(0)
    # C(100, 2) = 4950 tied combinations: beyond the largest pool (4096)
    geno, pheno = _copies(100, 500, seed=5)
    ds = epi.Dataset(ctx, geno, pheno)
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 2, 10, path=path)
    assert e.value.status == epi.EPI_EOVERFLOW
    # the context and the dataset stay usable
    geno2, pheno2 = random_data(40, 500, seed=6)
    r = epi.search(epi.Dataset(ctx, geno2, pheno2), 2, 10, path=path)
    oc, om, _ = O.search(geno2, pheno2, 2, 10)
    check_topn(r.combs, r.mi, oc, om)


def test_wait_limit_gives_etimeout_and_the_context_recovers(epi):
    ctx = epi.Context(0)
    geno, pheno = random_data(120, 4000, seed=7)
    ds = epi.Dataset(ctx, geno, pheno)
    want = epi.search(ds, 3, 20, path="popc")
    ctx.set_wait_limit(1000)
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 3, 20, path="tc")
    assert e.value.status == epi.EPI_ETIMEOUT
    ctx.set_wait_limit(0)
    got = epi.search(ds, 3, 20, path="tc")
    assert (got.combs == want.combs).all() and (got.mi == want.mi).all()


def test_injected_allocation_failure_gives_enomem(epi):
    ctx = epi.Context(0)
    geno, pheno = random_data(50, 600, seed=8)
    # the dataset's first allocation (the staging copy of the host inputs)
    ctx.inject_alloc_failure(0)
    with pytest.raises(epi.EpiError) as e:
        epi.Dataset(ctx, geno, pheno)
    assert e.value.status == epi.EPI_ENOMEM
    # a later allocation of the dataset (its genotype tables)
    ctx.inject_alloc_failure(2)
    with pytest.raises(epi.EpiError) as e:
        epi.Dataset(ctx, geno, pheno)
    assert e.value.status == epi.EPI_ENOMEM
    ds = epi.Dataset(ctx, geno, pheno)
    # the search's first allocation (its device output buffer)
    ctx.inject_alloc_failure(0)
    with pytest.raises(epi.EpiError) as e:
        epi.search(ds, 2, 10, path="popc")
    assert e.value.status == epi.EPI_ENOMEM
    for path in ("popc", "tc"):
        r = epi.search(ds, 2, 10, path=path)
        oc, om, _ = O.search(geno, pheno, 2, 10)
        check_topn(r.combs, r.mi, oc, om)
    # a cancelled injection never fires
    ctx.inject_alloc_failure(0)
    ctx.inject_alloc_failure(-1)
    assert len(epi.search(ds, 3, 5, path="tc")) == 5
