"""The allocation-free search entry point (epi_search_static).

It serves callers that cannot allocate device memory; it must return what
epi_search returns on the popcount path, call after call, although every call
reuses the same fixed device array, and it must refuse datasets too large for
that array before doing any work.
"""
import ctypes as C

import numpy as np
import pytest

from tests.helpers import F32_RTOL, F64_ATOL, random_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_02460_gb300 import epi
    lib = epi.load()
    fn = lib.epi_search_static
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return torch, epi, fn


def _run_static(torch, epi, fn, geno, pheno, k, top_n):
    g = torch.from_numpy(geno).cuda()
    p = torch.from_numpy(pheno).cuda()
    out = torch.zeros(top_n * epi.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros((top_n, 2, 3 ** k), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(g.data_ptr(), p.data_ptr(), geno.shape[0], geno.shape[1], int(pheno.sum()), k, top_n,
            out.data_ptr(), cnt.data_ptr(), n_out.data_ptr(), st.data_ptr(), stream)
    assert rc == 0, epi.load().epi_last_error()
    torch.cuda.synchronize()
    n = int(n_out.item())
    recs = np.frombuffer(out.cpu().numpy().tobytes(), dtype=epi.RESULT_DTYPE)[:n]
    return int(st.item()), recs, cnt.cpu().numpy().astype(np.uint32)[:n]


def test_static_search_matches_search_on_consecutive_calls(env):
    torch, epi, fn = env
    ctx = epi.Context(0)
    cases = [(3, 60, 1000, 50, 1), (2, 150, 777, 30, 2), (4, 24, 513, 40, 3), (3, 60, 1000, 50, 1)]
    for k, n, m, top_n, seed in cases:
        geno, pheno = random_data(n, m, seed=seed)
        want = epi.search(epi.Dataset(ctx, geno, pheno), k, top_n, path="popc")
        status, recs, counts = _run_static(torch, epi, fn, geno, pheno, k, top_n)
        assert status == 0
        assert len(recs) == len(want)
        assert (recs["snp"][:, :k].astype(np.int64) == want.combs).all()
        np.testing.assert_allclose(recs["mi"], want.mi, rtol=0, atol=F64_ATOL)
        assert (np.abs(recs["mi_f32"].astype(np.float64) - want.mi) <= F32_RTOL * want.mi + 1e-12).all()
        assert (counts == want.counts).all()


def test_static_search_reports_bad_inputs_and_refuses_large_datasets(env):
    torch, epi, fn = env
    # a larger dataset first, so that the shared array holds index entries
    # beyond what the small dataset below writes
    big_geno, big_pheno = random_data(40, 1500, seed=5)
    status, recs, _ = _run_static(torch, epi, fn, big_geno, big_pheno, 2, 10)
    assert status == 0 and len(recs) == 10
    geno, pheno = random_data(30, 200, seed=4)
    # n_cases that does not match the phenotype comes back as EPI_EINVAL with
    # no records (one more or one fewer than the true count; the genotype
    # reads stay inside this call's inputs either way)
    g = torch.from_numpy(geno).cuda()
    p = torch.from_numpy(pheno).cuda()
    out = torch.zeros(10 * epi.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for wrong in (int(pheno.sum()) + 1, int(pheno.sum()) - 1):
        n_out.fill_(7)
        rc = fn(g.data_ptr(), p.data_ptr(), 30, 200, wrong, 2, 10, out.data_ptr(), None,
                n_out.data_ptr(), st.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(st.item()) == epi.EPI_EINVAL
        assert int(n_out.item()) == 0
    # the array is usable again right after the rejected calls
    want = epi.search(epi.Dataset(epi.Context(0), geno, pheno), 2, 10, path="popc")
    status, recs, _ = _run_static(torch, epi, fn, geno, pheno, 2, 10)
    assert status == 0
    assert (recs["snp"][:, :2].astype(np.int64) == want.combs).all()
    # genotype tables larger than the fixed array: refused before any work
    big = torch.empty((12000, 16000), dtype=torch.uint8, device="cuda")
    bp = torch.zeros(16000, dtype=torch.uint8, device="cuda")
    rc = fn(big.data_ptr(), bp.data_ptr(), 12000, 16000, 0, 2, 10, out.data_ptr(), None, n_out.data_ptr(),
            st.data_ptr(), stream)
    assert rc == epi.EPI_EINVAL
    assert b"64 MiB" in epi.load().epi_last_error()
    # host pointers are refused
    rc = fn(geno.ctypes.data, pheno.ctypes.data, 30, 200, int(pheno.sum()), 2, 10, out.data_ptr(), None,
            n_out.data_ptr(), st.data_ptr(), stream)
    assert rc == epi.EPI_EINVAL
