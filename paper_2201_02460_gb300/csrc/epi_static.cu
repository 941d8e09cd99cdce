// Allocation-free variant of the popcount-path search.
//
// Some callers cannot allocate device memory: plug-ins running inside a host
// framework that owns every device allocation, or code with a fixed memory
// budget that must not grow at run time.  For them, epi_search_static runs the
// whole popcount search (genotype tables, exhaustive count and score, exact
// top-N) with every intermediate buffer carved out of one file-scope device
// array of fixed size, kStaticScratchBytes.  The caller passes device inputs
// and device outputs; the call performs no cudaMalloc, no cudaFree and no
// other allocating call.  Every GPU that loads the library holds the array
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "epi_host.h"
#include "epi_internal.cuh"

namespace epi {

// status message setter of the C-ABI (epi_api.cu)
void set_last_error(const char *msg);

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB

// The scratch array.  In host code its name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;

// What one device needs per call, resolved on the first call on that device
// (in the runtime's primary context of the device) and kept: the scratch
// array's device address and the two device attributes the launch plan uses.
struct DeviceSetup {
    unsigned char *scratch = nullptr;
    int num_sms = 0;
    int smem_optin = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

cudaError_t device_setup(int device, DeviceSetup *out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &S = g_setup[device];
    if (!S.scratch) {
        int sms = 0, optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        S.num_sms = sms;
        S.smem_optin = optin;
        S.scratch = static_cast<unsigned char *>(p);
    }
    *out = S;
    return cudaSuccess;
}

__global__ void check_cases_kernel(const int64_t *m1_dev, int64_t m1_given, int32_t *status)
{
    if (*m1_dev != m1_given) atomicOr(status, ST_BAD_PHENO);
}

// Invalid inputs leave no result: the record count is zeroed so that a caller
// reading n_out before status_dev sees an empty result.
__global__ void clear_on_bad_input_kernel(const int32_t *status, int32_t *n_out)
{
    if (*status & (ST_BAD_GENO | ST_BAD_PHENO)) *n_out = 0;
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += bytes;
        return at;
    }
};

bool is_dev(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

epi_status bad(epi_status s, const char *msg)
{
    set_last_error(msg);
    return s;
}

}  // namespace

}  // namespace epi

using namespace epi;

extern "C" epi_status epi_search_static(const uint8_t *geno_dev, const uint8_t *pheno_dev, int64_t n_snps,
                                        int64_t n_samples, int64_t n_cases, int order, int top_n,
                                        epi_result *out_dev, uint32_t *counts_dev, int32_t *n_out_dev,
                                        int32_t *status_dev, void *cuda_stream)
{
    if (!geno_dev || !pheno_dev || !out_dev || !n_out_dev || !status_dev)
        return bad(EPI_EINVAL, "epi_search_static: NULL pointer argument");
    if (n_snps < 1 || n_samples < 1 || n_samples > (1 << 23) - 1 || n_snps > (1 << 24))
        return bad(EPI_EINVAL, "epi_search_static: need 1 <= n_snps <= 2^24 and 1 <= n_samples < 2^23");
    if (n_cases < 0 || n_cases > n_samples) return bad(EPI_EINVAL, "epi_search_static: n_cases outside 0..n_samples");
    if (order < 1 || order > kMaxOrderTc || order > n_snps)
        return bad(EPI_EINVAL, "epi_search_static: order must lie in 1..min(5, n_snps)");
    if (top_n < 1 || top_n > 1024) return bad(EPI_EINVAL, "epi_search_static: top_n outside 1..1024");
    const uint64_t total = host_binom(n_snps, order);
    if (total >= ((uint64_t)1 << 62)) return bad(EPI_EUNSUPPORTED, "epi_search_static: too many combinations");

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return bad(EPI_ECUDA, "epi_search_static: no usable current device");
    if (!is_dev(geno_dev, device) || !is_dev(pheno_dev, device) || !is_dev(out_dev, device) ||
        !is_dev(n_out_dev, device) || !is_dev(status_dev, device) || (counts_dev && !is_dev(counts_dev, device)))
        return bad(EPI_EINVAL, "epi_search_static: inputs and outputs must be device memory of the current device");
    DeviceSetup setup;
    if (device_setup(device, &setup) != cudaSuccess)
        return bad(EPI_ECUDA, "epi_search_static: cannot read the device attributes or the scratch array's address");
    const int num_sms = setup.num_sms;
    const size_t smem_limit = (size_t)setup.smem_optin;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // layout of the dataset (Section 2.1) and of the search
    DevData d;
    d.n = n_snps; d.m = n_samples; d.m1 = n_cases; d.m0 = n_samples - n_cases;
    d.W1 = (int32_t)(((d.m1 + 127) / 128) * 4);
    d.W0 = (int32_t)(((d.m0 + 127) / 128) * 4);
    d.Wt = d.W1 + d.W0;
    const int k = order;
    int pool = top_n + 64 > 128 ? top_n + 64 : 128;
    pool = (pool + 31) & ~31;
    const int R = popc_default_row_group(k);
    const uint64_t span = total;
    int tile = 0, cand_p2 = 0, slots = 0, occ = 0;
    size_t smem = 0;
    int best = -1;
    for (int t : {512, 256, 128}) {
        if (t > 128 && (uint64_t)t * num_sms * 2 > span) continue;
        const int cp2 = next_pow2(pool + 2 * t);
        for (int s = 8; s >= 1; s--) {
            const size_t sm = popc_smem_bytes(k, d.Wt, s, cp2) + 1024;
            if (sm > smem_limit) continue;
            const int o = popc_max_active(k, R, sm);
            if (o <= 0) continue;
            const int score = (o < 8 ? o : 8) * 1000 + (t >= 256 ? 100 : 0) + s * 10 + (t == 512);
            if (score > best) { best = score; tile = t; cand_p2 = cp2; slots = s; smem = sm; occ = o; }
        }
    }
    if (best < 0) return bad(EPI_EUNSUPPORTED, "epi_search_static: a prefix table does not fit in shared memory");
    uint64_t grid64 = (uint64_t)num_sms * (uint64_t)occ;
    if (grid64 > (span + 127) / 128) grid64 = (span + 127) / 128;
    if (grid64 < 1) grid64 = 1;
    const int grid = (int)grid64;
    const int cells = [&] { int c = 1; for (int t = 0; t < k; t++) c *= 3; return c; }();

    Carve c;
    const size_t o_case = c.take((size_t)n_samples * 4);
    const size_t o_ctrl = c.take((size_t)n_samples * 4);
    const size_t o_m1 = c.take(8);
    const size_t o_status = c.take(8);     // status word, then the shared threshold word
    const size_t o_thr = o_status + 4;
    const size_t o_masks = c.take((size_t)n_snps * 3 * d.Wt * 4);
    const size_t o_binom = c.take((size_t)9 * (n_snps + 1) * 8);
    const size_t o_ls = c.take((size_t)grid * pool * 4);
    const size_t o_lr = c.take((size_t)grid * pool * 8);
    const size_t o_lc = c.take((size_t)grid * 4);
    const size_t o_cs = c.take((size_t)pool * 4);
    const size_t o_cr = c.take((size_t)pool * 8);
    const size_t o_cn = c.take(4);
    const size_t o_ct = c.take((size_t)pool * 2 * cells * 4);
    const size_t o_mi = c.take((size_t)pool * 8);
    const size_t o_cb = c.take((size_t)pool * k * 4);
    if (c.off > kStaticScratchBytes)
        return bad(EPI_EINVAL, "epi_search_static: dataset too large for the 64 MiB static scratch "
                               "(needs about n_snps * 3 * 2 * ceil(n_samples/128) * 16 bytes of genotype tables)");

    unsigned char *base = setup.scratch;
    cudaError_t e;
    int32_t *case_idx = reinterpret_cast<int32_t *>(base + o_case);
    int32_t *ctrl_idx = reinterpret_cast<int32_t *>(base + o_ctrl);
    int64_t *dm1 = reinterpret_cast<int64_t *>(base + o_m1);
    int32_t *status = reinterpret_cast<int32_t *>(base + o_status);
    uint32_t *thr = reinterpret_cast<uint32_t *>(base + o_thr);
    uint32_t *masks = reinterpret_cast<uint32_t *>(base + o_masks);
    uint64_t *binom = reinterpret_cast<uint64_t *>(base + o_binom);
    float *ls = reinterpret_cast<float *>(base + o_ls);
    uint64_t *lr = reinterpret_cast<uint64_t *>(base + o_lr);
    int32_t *lc = reinterpret_cast<int32_t *>(base + o_lc);
    float *cs = reinterpret_cast<float *>(base + o_cs);
    uint64_t *cr = reinterpret_cast<uint64_t *>(base + o_cr);
    int32_t *cn = reinterpret_cast<int32_t *>(base + o_cn);
    uint32_t *ct = reinterpret_cast<uint32_t *>(base + o_ct);
    double *mi = reinterpret_cast<double *>(base + o_mi);
    int32_t *cb = reinterpret_cast<int32_t *>(base + o_cb);
    d.masks = masks;
    d.binom = binom;

    // the array keeps whatever was there before (an earlier call, or memory
    // the device used before the library was loaded): the status word and the
    // shared threshold, adjacent, must start at zero; everything else is
    // written before it is read
    e = cudaMemsetAsync(base + o_status, 0, 8, st);
    if (e != cudaSuccess) return bad(EPI_ECUDA, "epi_search_static: cudaMemsetAsync failed");
    launch_scan_pheno(pheno_dev, n_samples, case_idx, ctrl_idx, dm1, status, st);
    check_cases_kernel<<<1, 1, 0, st>>>(dm1, n_cases, status);
    // the index maps hold exactly *dm1 cases and n_samples - *dm1 controls
    // written by this call; the pack kernel reads them only when that matches
    // n_cases (otherwise the search runs on all-zero rows and is reported as
    // EPI_EINVAL with no records)
    launch_pack_masks(geno_dev, n_snps, n_samples, case_idx, ctrl_idx, n_cases, d.W1, d.Wt, masks, status, num_sms, st,
                      dm1);
    launch_binom(n_snps, binom, num_sms, st);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_popc_search(d, k, R, 0, total, tile, pool, slots, cand_p2, thr, ls, lr, lc, grid, smem, st);
    if (e == cudaSuccess) e = launch_merge(ls, lr, lc, grid, pool, pool, cs, cr, cn, st);
    if (e == cudaSuccess) e = launch_rescore(d, k, pool, cr, cn, ct, mi, cb, st);
    if (e == cudaSuccess)
        e = launch_finalize(d, k, top_n, pool, cs, cr, cn, mi, cb, ct, thr, total, out_dev, counts_dev, n_out_dev,
                            status, st);
    if (e == cudaSuccess) {
        clear_on_bad_input_kernel<<<1, 1, 0, st>>>(status, n_out_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_publish_status(status, status_dev, st);
    if (e != cudaSuccess) return bad(EPI_ECUDA, cudaGetErrorString(e));
    return EPI_OK;
}
