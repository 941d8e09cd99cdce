// C-ABI of libepi: contexts, datasets and the search orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <map>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "epi_host.h"
#include "epi_internal.cuh"

using namespace epi;

struct epi_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    uint64_t launches = 0;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    int64_t live_datasets = 0;     // datasets created on this context and not yet destroyed
    // batched searches: device arena, pinned staging, one cached graph
    void *batch_dev = nullptr;
    size_t batch_dev_bytes = 0;
    void *batch_host = nullptr;
    size_t batch_host_bytes = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<uint64_t> batch_key;
    uint64_t next_dataset_id = 1;
    // autotuner choices by (order, SNP bucket, sample-word bucket)
    struct Tune { int R = 0, tile = 0, slots = 0, path = 0; double ms = 0; };
    std::map<uint64_t, Tune> tune;
    unsigned long long *waits_dev = nullptr;   // own buffer: per-role wait cycles of a profiled TC search
    int waits_grid = 0;                        // CTAs recorded in waits_dev (0: nothing recorded)
    bool destroy_requested = false;
    // test controls (epi_set_wait_limit, epi_inject_alloc_failure)
    unsigned long long wait_limit_ns = 0;   // tensor-core pipeline waits; 0 = the kernels' default
    int64_t fail_alloc_in = -1;             // device allocations until one fails; -1 = none
    bool tc_combined = true;                // epi_set_tc_variant: combined-class variant where it applies
};

struct epi_dataset {
    epi_ctx *ctx = nullptr;
    uint64_t id = 0;               // unique within the context (keys cached batch graphs)
    int64_t n = 0, m = 0, m1 = 0, m0 = 0;
    int32_t W1 = 0, W0 = 0, Wt = 0;
    uint32_t *masks = nullptr;
    uint64_t *binom = nullptr;
    unsigned char *b8 = nullptr;   // tensor-core operand (separate classes, E4M3), built on first use
    unsigned char *b8c = nullptr;  // the same for the combined-class variant (E5M2), built on first use
    float *lower[5] = {};          // exhaustive order-1..4 scores for the proposer, built on first use
    DevData dev() const
    {
        DevData d;
        d.n = n; d.m = m; d.m1 = m1; d.m0 = m0;
        d.W1 = W1; d.W0 = W0; d.Wt = Wt;
        d.masks = masks;
        d.binom = binom;
        return d;
    }
};

namespace {

thread_local std::string g_err;

epi_status fail(epi_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? EPI_ENOMEM : EPI_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

// Makes the context's device current for the scope of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// true when p is device (or managed) memory usable on `device`
bool is_device_ptr(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Every device allocation of a context's calls goes through these, so that a
// test can make the n-th one fail as an exhausted device would.
bool injected_alloc_failure(epi_ctx *ctx)
{
    if (ctx->fail_alloc_in < 0) return false;
    if (ctx->fail_alloc_in == 0) {
        ctx->fail_alloc_in = -1;
        return true;
    }
    ctx->fail_alloc_in--;
    return false;
}

cudaError_t ctx_malloc(epi_ctx *ctx, void **p, size_t bytes)
{
    if (injected_alloc_failure(ctx)) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t ctx_malloc_async(epi_ctx *ctx, void **p, size_t bytes, cudaStream_t st)
{
    if (injected_alloc_failure(ctx)) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, st);
}

int pow3i(int k)
{
    int r = 1;
    while (k-- > 0) r *= 3;
    return r;
}

// Carves aligned pieces out of the context's scratch arena.
struct Arena {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += count * sizeof(T);
        return at;
    }
};

epi_status ensure_scratch(epi_ctx *ctx, size_t bytes)
{
    if (ctx->scratch_bytes >= bytes) return EPI_OK;
    if (ctx->scratch) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    want = (want + ((1u << 20) - 1)) & ~(size_t)((1u << 20) - 1);
    CK(ctx_malloc(ctx, &ctx->scratch, want));
    ctx->scratch_bytes = want;
    return EPI_OK;
}

// Size bucket of the autotuner: order, log2 of the SNP count, log2 of the
// sample words (choices transfer between datasets of similar shape).
uint64_t tune_key(int k, int64_t n, int32_t wt)
{
    int nb = 0, wb = 0;
    while ((int64_t)1 << (nb + 1) <= n) nb++;
    while ((1 << (wb + 1)) <= wt) wb++;
    return ((uint64_t)k << 48) | ((uint64_t)nb << 24) | (uint64_t)wb;
}

struct SearchPlan {
    int k = 0, top_n = 0, pool = 0, tile = 0, slots = 0, cand_p2 = 0, grid = 0, R = 0;
    bool tc = false;
    int comb_p = 0;                // tensor path: class shift of the combined-class variant, 0 = separate classes
    bool global_prefix = false;    // popcount path: prefix tables in a global buffer (orders 7-8)
    bool pair = false;             // popcount path: the (k-2)-prefix kernel (orders 6-8)
    float *all_scores = nullptr;   // optional: every combination's score (popcount path)
    size_t smem = 0;
    uint64_t rb = 0, re = 0, total = 0;
};

// Prefixes staged per sub-tile when the prefix tables live in global memory
// (orders 7-8; tuning parameter: 1, 2 and 4 measured 170, 131 and 210 ms on
// the order-8 Table-2 workload).
#ifndef EPI_GP_SLOTS
#define EPI_GP_SLOTS 2
#endif
constexpr int kGlobalPrefixSlots = EPI_GP_SLOTS;

// Popcount-path launch shape: row group R (counters per thread), sub-tile T,
// staged prefixes per sub-tile and CTAs per SM.  Residency first (the POPC
// pipe needs many warps to hide its latency), then staged prefixes.
epi_status plan_popc(const epi_dataset *ds, SearchPlan &p, int R_req = 0)
{
    const epi_ctx *ctx = ds->ctx;
    const uint64_t span = p.re - p.rb;
    p.R = R_req ? R_req : popc_default_row_group(p.k);
    if (!popc_row_group_ok(p.k, p.R)) return fail(EPI_EINVAL, "row group %d invalid for order %d", p.R, p.k);
    const size_t limit = ctx->smem_optin ? ctx->smem_optin : 227 * 1024;
    int best_score = -1;
    // an autotuned shape for this size bucket, unless the caller forces one
    int tune_tile = 0, tune_slots = 0;
    if (!R_req) {
        auto it = ctx->tune.find(tune_key(p.k, ds->n, ds->Wt));
        if (it != ctx->tune.end() && it->second.R) {
            p.R = it->second.R;
            tune_tile = it->second.tile;
            tune_slots = it->second.slots;
        }
    } else if (p.tile && p.slots) {
        tune_tile = p.tile;
        tune_slots = p.slots;
    }
    for (int tile : {512, 256, 128}) {
        // small searches: keep every CTA busy
        if (tile > 128 && (uint64_t)tile * ctx->num_sms * 2 > span && tile != tune_tile) continue;
        if (tune_tile && tile != tune_tile) continue;
        const int cand_p2 = next_pow2(p.pool + 2 * tile);
        for (int s = 8; s >= 1; s--) {
            if (tune_slots && s != tune_slots) continue;
            const size_t sm = popc_smem_bytes(p.k, ds->Wt, s, cand_p2) + 1024;
            if (sm > limit) continue;
            const int occ = popc_max_active(p.k, p.R, sm);
            if (occ <= 0) continue;
            // sub-tiles of 128 combinations: the autotuner's choice on every
            // measured workload (orders 2-5, 1600-16000 samples: 4-27 %
            // faster than 512)
            const int score = std::min(occ, 8) * 1000 + (tile == 128 ? 100 : 0) + s * 10 + (tile == 256);
            if (score > best_score) {
                best_score = score;
                p.tile = tile; p.cand_p2 = cand_p2; p.slots = s; p.smem = sm; p.grid = occ;
            }
        }
    }
    p.global_prefix = false;
    if (popc_global_prefix_ok(p.k, p.R)) {
        // orders 7-8: the prefix tables (729 or 2187 rows) go to per-CTA
        // global buffers (the CTA's threads walk the same rows, shared
        // through L1/L2).  In shared memory one table leaves room for one or
        // two CTAs per SM; with global tables up to four run (the register
        // limit), measured 1.5-1.7x faster at 2048 individuals
        best_score = -1;
        for (int tile : {256, 128}) {
            if (tune_tile && tile != tune_tile) continue;
            const int cand_p2 = next_pow2(p.pool + 2 * tile);
            const size_t sm = popc_smem_bytes(p.k, ds->Wt, kGlobalPrefixSlots, cand_p2, true) + 1024;
            if (sm > limit) continue;
            const int occ = popc_max_active(p.k, p.R, sm, true);
            if (occ <= 0) continue;
            p.tile = tile; p.cand_p2 = cand_p2; p.slots = kGlobalPrefixSlots; p.smem = sm; p.grid = std::min(occ, 4);
            p.global_prefix = true;
            best_score = 0;
            break;
        }
    }
    if (best_score < 0)
        return fail(EPI_EUNSUPPORTED, "order %d with %lld samples: one prefix table does not fit in shared memory",
                    p.k, (long long)ds->m);
    uint64_t grid = (uint64_t)ctx->num_sms * (uint64_t)p.grid;
    // orders 6-8: the (k-2)-prefix kernel, one 1024-thread CTA per SM, its
    // own number of waves
    p.pair = popc_pair_applies(p.k, ds->Wt, p.pool, p.all_scores != nullptr);
    if (p.pair) {
        p.global_prefix = false;
        grid = (uint64_t)popc_pair_grid(ctx->num_sms, p.k, ds->n);
    }
    const uint64_t by_work = (span + 127) / 128;
    if (grid > by_work) grid = by_work;
    if (grid < 1) grid = 1;
    p.grid = (int)grid;
    return EPI_OK;
}

// Tensor-core path conditions: orders 2..5, both classes present.  A rank
// range is searched over whole first-SNP blocks and clipped in the epilogue.
bool tc_applicable(const epi_dataset *ds, int k, uint64_t rb, uint64_t re, uint64_t total)
{
    (void)rb; (void)re; (void)total;
    return k >= 2 && k <= 5 && ds->m1 > 0 && ds->m0 > 0 && ds->n >= k + 1;
}

epi_status choose_path(const epi_dataset *ds, int k, int path, uint64_t rb, uint64_t re, uint64_t total, bool &tc)
{
    const bool ok = tc_applicable(ds, k, rb, re, total);
    if (path == EPI_PATH_TC) {
        if (!ok)
            return fail(EPI_EUNSUPPORTED,
                        "tensor-core path needs order 2..5, cases and controls, and the whole combination range");
        tc = true;
    } else if (path == EPI_PATH_POPC) {
        tc = false;
    } else {
        // automatic choice: the tensor path counts whole first-SNP blocks, so
        // it is taken for a rank range only when that adds at most as much
        // work again as the range itself
        tc = ok && k >= 3 && (re - rb == total || tc_range_work(ds->n, k, rb, re) <= 2 * (re - rb));
        auto it = ds->ctx->tune.find(tune_key(k, ds->n, ds->Wt));
        if (ok && it != ds->ctx->tune.end() && it->second.path) tc = it->second.path == EPI_PATH_TC;
    }
    return EPI_OK;
}

// The dataset's B operand for a class shift (0: separate-class variant).
epi_status ensure_b8(epi_dataset *ds, int comb_p = 0)
{
    unsigned char *&buf = comb_p ? ds->b8c : ds->b8;
    if (buf) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    CK(ctx_malloc(ctx, (void **)&buf, tc_b8_bytes(ds->dev())));
    CK(launch_build_b8(ds->dev(), buf, ctx->num_sms, ctx->stream, comb_p));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status make_plan(const epi_dataset *ds, SearchPlan &p, int path)
{
    epi_status st = choose_path(ds, p.k, path, p.rb, p.re, p.total, p.tc);
    if (st != EPI_OK) return st;
    if (!p.tc) return plan_popc(ds, p);
    p.grid = ds->ctx->num_sms;
    p.comb_p = ds->ctx->tc_combined ? tc_comb_shift(ds->dev(), p.k) : 0;
    return EPI_OK;
}

// Queues one search pass with the given plan; results land in device memory.
epi_status queue_search(epi_dataset *ds, const SearchPlan &p, int path, epi_result *out_dev, uint32_t *counts_dev,
                        int32_t *n_out_dev, int32_t **status_dev_out, uint32_t *dump = nullptr)
{
    epi_ctx *ctx = ds->ctx;
    (void)path;
    const int cells = pow3i(p.k);
    Arena a;
    const size_t o_thr = a.take<uint32_t>(1);
    const size_t o_status = a.take<int32_t>(1);
    const size_t o_ls = a.take<float>((size_t)p.grid * p.pool);
    const size_t o_lr = a.take<uint64_t>((size_t)p.grid * p.pool);
    const size_t o_lc = a.take<int32_t>((size_t)p.grid);
    const size_t o_cs = a.take<float>((size_t)p.pool);
    const size_t o_cr = a.take<uint64_t>((size_t)p.pool);
    const size_t o_cn = a.take<int32_t>(1);
    const size_t o_ct = a.take<uint32_t>((size_t)p.pool * 2 * cells);
    const size_t o_mi = a.take<double>((size_t)p.pool);
    const size_t o_cb = a.take<int32_t>((size_t)p.pool * p.k);
    const size_t o_ic = a.take<uint64_t>(2 * ((size_t)ds->n + 1));
    const size_t o_pre =
        p.global_prefix ? a.take<uint32_t>((size_t)p.grid * p.slots * popc_slot_words(p.k, ds->Wt)) : 0;
    const size_t o_sing = p.pair ? a.take<uint32_t>((size_t)p.grid * popc_pair_sing_words(p.k, ds->n)) : 0;
    // tensor path: candidate buffers in global memory when they do not fit
    // beside the operand rings in shared memory (large pools)
    const int tc_cp2 = p.tc ? tc_cand_p2(p.k, p.pool, p.comb_p != 0) : 0;
    const bool tc_cg = p.tc && tc_smem_bytes(tc_cp2, p.k, false, p.comb_p != 0) > ctx->smem_optin;
    const size_t o_tcs = tc_cg ? a.take<float>((size_t)p.grid * tc_cp2) : 0;
    const size_t o_tcr = tc_cg ? a.take<uint64_t>((size_t)p.grid * tc_cp2) : 0;
    epi_status st = ensure_scratch(ctx, a.off);
    if (st != EPI_OK) return st;
    char *base = static_cast<char *>(ctx->scratch);
    uint32_t *thr = reinterpret_cast<uint32_t *>(base + o_thr);
    int32_t *status = reinterpret_cast<int32_t *>(base + o_status);
    float *ls = reinterpret_cast<float *>(base + o_ls);
    uint64_t *lr = reinterpret_cast<uint64_t *>(base + o_lr);
    int32_t *lc = reinterpret_cast<int32_t *>(base + o_lc);
    float *cs = reinterpret_cast<float *>(base + o_cs);
    uint64_t *cr = reinterpret_cast<uint64_t *>(base + o_cr);
    int32_t *cn = reinterpret_cast<int32_t *>(base + o_cn);
    uint32_t *ct = reinterpret_cast<uint32_t *>(base + o_ct);
    double *mi = reinterpret_cast<double *>(base + o_mi);
    int32_t *cb = reinterpret_cast<int32_t *>(base + o_cb);
    uint64_t *ic = reinterpret_cast<uint64_t *>(base + o_ic);
    if (p.tc) {
        st = ensure_b8(ds, p.comb_p);
        if (st != EPI_OK) return st;
    }
    // threshold word and status word live in the first 512 bytes
    CK(cudaMemsetAsync(base, 0, 512, ctx->stream));
    const DevData d = ds->dev();
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (ctx->profiling) {
        CK(cudaEventCreate(&ev0));
        CK(cudaEventCreate(&ev1));
        ctx->prof_events.emplace_back(ev0, ev1);
        CK(cudaEventRecord(ev0, ctx->stream));
    }
    if (p.tc) {
        int cand_p2 = 0;
        unsigned long long *waits = nullptr;
        if (ctx->profiling) {
            if (!ctx->waits_dev)
                CK(cudaMalloc((void **)&ctx->waits_dev, (size_t)ctx->num_sms * kTcWaitSlots * 8));
            CK(cudaMemsetAsync(ctx->waits_dev, 0, (size_t)p.grid * kTcWaitSlots * 8, ctx->stream));
            waits = ctx->waits_dev;
            ctx->waits_grid = p.grid;
        }
        CK(launch_tc_search(d, p.k, p.comb_p ? ds->b8c : ds->b8, ic, p.pool, thr, ls, lr, lc, status, p.grid,
                            p.total, p.rb, p.re, ctx->stream, &cand_p2,
                            tc_cg ? reinterpret_cast<float *>(base + o_tcs) : nullptr,
                            tc_cg ? reinterpret_cast<uint64_t *>(base + o_tcr) : nullptr, dump, waits,
                            ctx->wait_limit_ns, p.comb_p));
        ctx->launches += 1;   // item table
    } else {
        CK(launch_popc_search(d, p.k, p.R, p.rb, p.re, p.tile, p.pool, p.slots, p.cand_p2, thr, ls, lr, lc, p.grid,
                              p.smem, ctx->stream, p.all_scores,
                              p.global_prefix ? reinterpret_cast<uint32_t *>(base + o_pre) : nullptr,
                              p.pair ? reinterpret_cast<uint32_t *>(base + o_sing) : nullptr, p.top_n));
    }
    if (ev1) CK(cudaEventRecord(ev1, ctx->stream));
    CK(launch_merge(ls, lr, lc, p.grid, p.pool, p.pool, cs, cr, cn, ctx->stream));
    CK(launch_rescore(d, p.k, p.pool, cr, cn, ct, mi, cb, ctx->stream));
    CK(launch_finalize(d, p.k, p.top_n, p.pool, cs, cr, cn, mi, cb, ct, thr, p.re - p.rb, out_dev, counts_dev,
                       n_out_dev, status, ctx->stream));
    ctx->launches += 4;
    *status_dev_out = status;
    return EPI_OK;
}

epi_status check_search_args(epi_dataset *ds, int order, int top_n, int path, uint64_t rb, uint64_t &re,
                             uint64_t &total)
{
    if (!ds) return fail(EPI_EINVAL, "dataset is NULL");
    if (order < 1 || order > EPI_MAX_ORDER) return fail(EPI_EINVAL, "order %d outside 1..%d", order, EPI_MAX_ORDER);
    if (order > ds->n) return fail(EPI_EINVAL, "order %d exceeds the %lld SNPs", order, (long long)ds->n);
    if (top_n < 1 || top_n > 1024) return fail(EPI_EINVAL, "top_n %d outside 1..1024", top_n);
    if (path < EPI_PATH_AUTO || path > EPI_PATH_TC) return fail(EPI_EINVAL, "unknown path %d", path);
    if (order > kMaxOrderGpu) return fail(EPI_EUNSUPPORTED, "order %d: the GPU search covers orders 1..%d", order,
                                          kMaxOrderGpu);
    total = host_binom(ds->n, order);
    if (total >= ((uint64_t)1 << 62)) return fail(EPI_EUNSUPPORTED, "C(%lld, %d) is too large", (long long)ds->n, order);
    if (re > total) re = total;
    if (rb > re) rb = re;
    (void)rb;
    return EPI_OK;
}

int initial_pool(int top_n)
{
    int p = std::max(top_n + 64, 128);
    return (p + 31) & ~31;
}

constexpr int kMaxPool = 4096;

epi_status run_search_sync(epi_dataset *ds, int order, int top_n, int path, uint64_t rb, uint64_t re,
                           epi_result *out, uint32_t *counts, int *n_out)
{
    uint64_t total = 0;
    epi_status st = check_search_args(ds, order, top_n, path, rb, re, total);
    if (st != EPI_OK) return st;
    if (!out || !n_out) return fail(EPI_EINVAL, "out and n_out must not be NULL");
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    *n_out = 0;
    if (rb >= re) return EPI_OK;
    const int cells = pow3i(order);
    int pool = initial_pool(top_n);
    for (;;) {
        SearchPlan p;
        p.k = order; p.top_n = top_n; p.pool = pool; p.rb = rb; p.re = re; p.total = total;
        st = make_plan(ds, p, path);
        if (st != EPI_OK) return st;
        // device-side outputs of this pass (stream-ordered allocation)
        const size_t rec_b = ((size_t)top_n * sizeof(epi_result) + 255) & ~(size_t)255;
        const size_t cnt_b = ((size_t)top_n * 2 * cells * 4 + 255) & ~(size_t)255;
        void *dout = nullptr;
        CK(ctx_malloc_async(ctx, &dout, rec_b + cnt_b + 256, ctx->stream));
        epi_result *out_dev = static_cast<epi_result *>(dout);
        uint32_t *cnt_dev = reinterpret_cast<uint32_t *>(static_cast<char *>(dout) + rec_b);
        int32_t *nout_dev = reinterpret_cast<int32_t *>(static_cast<char *>(dout) + rec_b + cnt_b);
        int32_t *status_dev = nullptr;
        st = queue_search(ds, p, path, out_dev, counts ? cnt_dev : nullptr, nout_dev, &status_dev);
        if (st != EPI_OK) { cudaFreeAsync(dout, ctx->stream); return st; }
        int32_t hst[2] = {0, 0};
        CK(cudaMemcpyAsync(&hst[0], status_dev, 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&hst[1], nout_dev, 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (hst[0] & ST_POOL_OVERFLOW) {
            cudaFreeAsync(dout, ctx->stream);
            if (pool >= kMaxPool)
                return fail(EPI_EOVERFLOW, "candidate pool of %d cannot prove the exact top %d (ties)", pool, top_n);
            pool = std::min(pool * 4, kMaxPool);
            continue;
        }
        if (hst[0] & ST_TIMEOUT) { cudaFreeAsync(dout, ctx->stream); return fail(EPI_ETIMEOUT, "device wait expired"); }
        if (hst[0] != 0) { cudaFreeAsync(dout, ctx->stream); return fail(EPI_ECUDA, "device status 0x%x", hst[0]); }
        const int n = hst[1];
        CK(cudaMemcpyAsync(out, out_dev, (size_t)n * sizeof(epi_result), cudaMemcpyDeviceToHost, ctx->stream));
        if (counts)
            CK(cudaMemcpyAsync(counts, cnt_dev, (size_t)n * 2 * cells * 4, cudaMemcpyDeviceToHost, ctx->stream));
        cudaFreeAsync(dout, ctx->stream);
        CK(cudaStreamSynchronize(ctx->stream));
        *n_out = n;
        return EPI_OK;
    }
}

}  // namespace

namespace epi {
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace epi


namespace {

// One dataset of a batched search and where its buffers live.
struct BatchItem {
    epi_dataset *ds = nullptr;
    int k = 0, top_n = 0, pool = 0, cells = 0;
    bool tc = false;
    uint64_t total = 0;
    double cost = 0;
    int group = -1, cta_begin = 0, cta_count = 0;
    // device offsets in the batch arena
    size_t o_thr = 0, o_status = 0, o_code = 0, o_nout = 0, o_cs = 0, o_cr = 0, o_cn = 0, o_ct = 0, o_mi = 0,
           o_cb = 0, o_ic = 0, o_rec = 0, o_cnt = 0, o_ls = 0, o_lr = 0, o_lc = 0;
    // pinned host offsets of the copied-back results
    size_t h_rec = 0, h_cnt = 0, h_nout = 0, h_code = 0;
};

struct BatchGroup {
    bool tc = false;
    int k = 0, R = 0, tile = 0, slots = 0, cand_p2 = 0, pool = 0, max_wt = 0, grid = 0;
    int64_t max_n = 0;
    size_t smem = 0;
    std::vector<int> items;
    size_t o_desc = 0, o_tmap = 0, o_ctads = 0, o_ls = 0, o_lr = 0, o_lc = 0;
    size_t o_tcs = 0, o_tcr = 0;   // tensor path: global candidate buffers (0: in shared memory)
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Popcount launch shape for a group: residency first, then staged prefixes.
bool plan_group_popc(const epi_ctx *ctx, BatchGroup &g)
{
    const size_t limit = ctx->smem_optin ? ctx->smem_optin : 227 * 1024;
    g.R = popc_default_row_group(g.k);
    int t_tile = 0, t_slots = 0;
    auto tn = ctx->tune.find(tune_key(g.k, g.max_n, g.max_wt));
    if (tn != ctx->tune.end() && tn->second.R) { g.R = tn->second.R; t_tile = tn->second.tile; t_slots = tn->second.slots; }
    int best = -1;
    for (int tile : {512, 256, 128}) {
        if (t_tile ? tile != t_tile : tile == 128) continue;
        const int cp2 = next_pow2(g.pool + 2 * tile);
        for (int sl = 8; sl >= 1; sl--) {
            if (t_slots && sl != t_slots) continue;
            const size_t sm = popc_smem_bytes(g.k, g.max_wt, sl, cp2) + 1024;
            if (sm > limit) continue;
            const int occ = popc_max_active(g.k, g.R, sm);
            if (occ <= 0) continue;
            const int score = std::min(occ, 8) * 1000 + sl * 10 + (tile == 512);
            if (score > best) { best = score; g.tile = tile; g.cand_p2 = cp2; g.slots = sl; g.smem = sm; g.grid = occ; }
        }
    }
    if (best < 0) return false;
    g.grid *= ctx->num_sms;
    return true;
}

// CTAs of a group's grid spread over its datasets in proportion to work.
void split_ctas(BatchGroup &g, std::vector<BatchItem> &items)
{
    const int n = (int)g.items.size();
    if (g.grid < n) g.grid = n;
    double total = 0;
    for (int i : g.items) total += items[i].cost;
    int used = 0;
    std::vector<double> frac(n);
    for (int q = 0; q < n; q++) {
        BatchItem &it = items[g.items[q]];
        const double share = total > 0 ? it.cost / total * (double)(g.grid - n) : 0.0;
        it.cta_count = 1 + (int)share;
        frac[q] = share - (double)(int)share;
        used += it.cta_count;
    }
    // hand out the remainder by largest fractional share
    std::vector<int> order(n);
    for (int q = 0; q < n; q++) order[q] = q;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return frac[a] > frac[b]; });
    for (int q = 0; used < g.grid; q = (q + 1) % n, used++) items[g.items[order[q]]].cta_count++;
    int at = 0;
    for (int q = 0; q < n; q++) {
        BatchItem &it = items[g.items[q]];
        it.cta_begin = at;
        at += it.cta_count;
    }
}

epi_status ensure_batch_buffers(epi_ctx *ctx, size_t dev_bytes, size_t host_bytes)
{
    if (ctx->batch_dev_bytes < dev_bytes || ctx->batch_host_bytes < host_bytes) {
        if (ctx->batch_exec) { cudaGraphExecDestroy(ctx->batch_exec); ctx->batch_exec = nullptr; }
        ctx->batch_key.clear();
    }
    if (ctx->batch_dev_bytes < dev_bytes) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->batch_dev) cudaFree(ctx->batch_dev);
        ctx->batch_dev = nullptr;
        ctx->batch_dev_bytes = 0;
        CK(ctx_malloc(ctx, &ctx->batch_dev, dev_bytes));
        ctx->batch_dev_bytes = dev_bytes;
    }
    if (ctx->batch_host_bytes < host_bytes) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
        ctx->batch_host = nullptr;
        ctx->batch_host_bytes = 0;
        CK(cudaMallocHost(&ctx->batch_host, host_bytes));
        ctx->batch_host_bytes = host_bytes;
    }
    if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    return EPI_OK;
}

// Records every step of the batched search on `st` (captured into a graph).
epi_status record_batch(epi_ctx *ctx, std::vector<BatchItem> &items, std::vector<BatchGroup> &groups, cudaStream_t st)
{
    char *dev = static_cast<char *>(ctx->batch_dev);
    char *host = static_cast<char *>(ctx->batch_host);
    // thresholds and status words of all datasets sit in one block at offset 0
    CK(cudaMemsetAsync(dev, 0, items.size() * 256, st));
    for (auto &g : groups) {
        if (g.tc)
            for (int i : g.items)
                CK(launch_tc_item_cum(items[i].ds->dev(), g.k, 0, items[i].total,
                                      reinterpret_cast<uint64_t *>(dev + items[i].o_ic), st));
        float *ls = reinterpret_cast<float *>(dev + g.o_ls);
        uint64_t *lr = reinterpret_cast<uint64_t *>(dev + g.o_lr);
        int32_t *lc = reinterpret_cast<int32_t *>(dev + g.o_lc);
        int32_t *ctads = reinterpret_cast<int32_t *>(dev + g.o_ctads);
        // every CTA of a TC group reports a timeout through its dataset's status
        if (g.tc)
            CK(launch_tc_batch(dev + g.o_desc, ctads, g.k, g.pool, ls, lr, lc,
                               reinterpret_cast<int32_t *>(dev + items[g.items[0]].o_status), g.grid, st,
                               g.o_tcs ? reinterpret_cast<float *>(dev + g.o_tcs) : nullptr,
                               g.o_tcs ? reinterpret_cast<uint64_t *>(dev + g.o_tcr) : nullptr));
        else
            CK(launch_popc_batch(dev + g.o_desc, ctads, g.k, g.R, g.max_wt, g.tile, g.pool, g.slots, g.cand_p2, ls, lr,
                                 lc, g.grid, g.smem, st));
        ctx->launches += 1;
    }
    for (auto &it : items) {
        const BatchGroup &g = groups[it.group];
        const DevData d = it.ds->dev();
        float *ls = reinterpret_cast<float *>(dev + g.o_ls) + (size_t)it.cta_begin * g.pool;
        uint64_t *lr = reinterpret_cast<uint64_t *>(dev + g.o_lr) + (size_t)it.cta_begin * g.pool;
        int32_t *lc = reinterpret_cast<int32_t *>(dev + g.o_lc) + it.cta_begin;
        float *cs = reinterpret_cast<float *>(dev + it.o_cs);
        uint64_t *cr = reinterpret_cast<uint64_t *>(dev + it.o_cr);
        int32_t *cn = reinterpret_cast<int32_t *>(dev + it.o_cn);
        uint32_t *ct = reinterpret_cast<uint32_t *>(dev + it.o_ct);
        double *mi = reinterpret_cast<double *>(dev + it.o_mi);
        int32_t *cb = reinterpret_cast<int32_t *>(dev + it.o_cb);
        uint32_t *thr = reinterpret_cast<uint32_t *>(dev + it.o_thr);
        int32_t *status = reinterpret_cast<int32_t *>(dev + it.o_status);
        epi_result *rec = reinterpret_cast<epi_result *>(dev + it.o_rec);
        uint32_t *cnt = reinterpret_cast<uint32_t *>(dev + it.o_cnt);
        int32_t *nout = reinterpret_cast<int32_t *>(dev + it.o_nout);
        int32_t *code = reinterpret_cast<int32_t *>(dev + it.o_code);
        CK(launch_merge(ls, lr, lc, it.cta_count, g.pool, it.pool, cs, cr, cn, st));
        CK(launch_rescore(d, it.k, it.pool, cr, cn, ct, mi, cb, st));
        CK(launch_finalize(d, it.k, it.top_n, it.pool, cs, cr, cn, mi, cb, ct, thr, it.total, rec, cnt, nout, status,
                           st));
        CK(launch_publish_status(status, code, st));
        ctx->launches += 4;
        CK(cudaMemcpyAsync(host + it.h_rec, rec, (size_t)it.top_n * sizeof(epi_result), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(host + it.h_cnt, cnt, (size_t)it.top_n * 2 * it.cells * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(host + it.h_nout, nout, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(host + it.h_code, code, 4, cudaMemcpyDeviceToHost, st));
    }
    return EPI_OK;
}

}  // namespace

extern "C" epi_status epi_search_batched(epi_ctx *ctx, epi_dataset *const *dss, const int *orders, const int *top_ns,
                                         int n_ds, int path, epi_result *const *outs, uint32_t *const *counts,
                                         int *n_outs)
{
    if (!ctx || !dss || !orders || !top_ns || !outs || !n_outs) return fail(EPI_EINVAL, "NULL argument");
    if (n_ds < 1 || n_ds > 4096) return fail(EPI_EINVAL, "n_ds %d outside 1..4096", n_ds);
    std::vector<BatchItem> items((size_t)n_ds);
    for (int i = 0; i < n_ds; i++) {
        BatchItem &it = items[i];
        it.ds = dss[i];
        if (!it.ds || it.ds->ctx != ctx) return fail(EPI_EINVAL, "dataset %d is NULL or belongs to another context", i);
        if (!outs[i]) return fail(EPI_EINVAL, "outs[%d] is NULL", i);
        uint64_t re = UINT64_MAX, total = 0;
        epi_status st = check_search_args(it.ds, orders[i], top_ns[i], path, 0, re, total);
        if (st != EPI_OK) return fail(st, "dataset %d: %s", i, epi_last_error());
        it.k = orders[i];
        it.top_n = top_ns[i];
        it.total = total;
        it.pool = initial_pool(it.top_n);
        it.cells = pow3i(it.k);
        st = choose_path(it.ds, it.k, path, 0, total, total, it.tc);
        if (st != EPI_OK) return fail(st, "dataset %d: %s", i, epi_last_error());
        const DevData d = it.ds->dev();
        // work estimate for the CTA split: a tensor-core item costs its K stages,
        // but never less than its epilogue (about 32 stages' worth)
        it.cost = it.tc ? (double)tc_item_count(d.n, it.k) * (double)std::max(d.Wt / 4, 32)
                        : (double)total * (double)(it.cells / 3) * (double)d.Wt;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    // one group per (path, order)
    std::vector<BatchGroup> groups;
    for (int i = 0; i < n_ds; i++) {
        int gi = -1;
        for (size_t q = 0; q < groups.size(); q++)
            if (groups[q].tc == items[i].tc && groups[q].k == items[i].k) gi = (int)q;
        if (gi < 0) {
            groups.emplace_back();
            gi = (int)groups.size() - 1;
            groups[gi].tc = items[i].tc;
            groups[gi].k = items[i].k;
        }
        items[i].group = gi;
        BatchGroup &g = groups[gi];
        g.items.push_back(i);
        g.pool = std::max(g.pool, items[i].pool);
        g.max_wt = std::max(g.max_wt, items[i].ds->Wt);
        g.max_n = std::max(g.max_n, items[i].ds->n);
    }
    for (auto &g : groups) {
        if (g.tc) g.grid = ctx->num_sms;
        else if (!plan_group_popc(ctx, g))
            return fail(EPI_EUNSUPPORTED, "order %d: a prefix table of the largest dataset does not fit in shared memory", g.k);
        split_ctas(g, items);
    }
    // device arena: per-dataset threshold/status block first, then buffers
    Arena a;
    for (auto &it : items) {
        const size_t base = a.take<char>(256);
        it.o_thr = base;
        it.o_status = base + 4;
        it.o_code = base + 8;
        it.o_nout = base + 12;
    }
    for (auto &g : groups) {
        g.o_desc = a.take<char>((g.tc ? tc_ds_bytes() : popc_ds_bytes()) * g.items.size());
        g.o_tmap = a.take<char>((size_t)128 * g.items.size());
        g.o_ctads = a.take<int32_t>((size_t)g.grid);
        g.o_ls = a.take<float>((size_t)g.grid * g.pool);
        g.o_lr = a.take<uint64_t>((size_t)g.grid * g.pool);
        g.o_lc = a.take<int32_t>((size_t)g.grid);
        if (g.tc && tc_smem_bytes(tc_cand_p2(g.k, g.pool), g.k, false) > ctx->smem_optin) {
            g.o_tcs = a.take<float>((size_t)g.grid * tc_cand_p2(g.k, g.pool));
            g.o_tcr = a.take<uint64_t>((size_t)g.grid * tc_cand_p2(g.k, g.pool));
        }
    }
    for (auto &it : items) {
        it.o_cs = a.take<float>((size_t)it.pool);
        it.o_cr = a.take<uint64_t>((size_t)it.pool);
        it.o_cn = a.take<int32_t>(1);
        it.o_ct = a.take<uint32_t>((size_t)it.pool * 2 * it.cells);
        it.o_mi = a.take<double>((size_t)it.pool);
        it.o_cb = a.take<int32_t>((size_t)it.pool * it.k);
        it.o_ic = a.take<uint64_t>(2 * ((size_t)it.ds->n + 1));
        it.o_rec = a.take<epi_result>((size_t)it.top_n);
        it.o_cnt = a.take<uint32_t>((size_t)it.top_n * 2 * it.cells);
    }
    size_t hoff = 0;
    for (auto &it : items) {
        it.h_rec = hoff; hoff = align_up(hoff + (size_t)it.top_n * sizeof(epi_result), 64);
        it.h_cnt = hoff; hoff = align_up(hoff + (size_t)it.top_n * 2 * it.cells * 4, 64);
        it.h_nout = hoff; hoff += 64;
        it.h_code = hoff; hoff += 64;
    }
    // descriptors are staged after the results in the pinned buffer
    size_t hdesc = hoff;
    for (auto &g : groups) hdesc = align_up(hdesc + (g.tc ? tc_ds_bytes() : popc_ds_bytes()) * g.items.size() +
                                            128 * g.items.size() + (size_t)g.grid * 4, 256);
    epi_status st = ensure_batch_buffers(ctx, a.off, hdesc + 256);
    if (st != EPI_OK) return st;
    for (auto &it : items)
        if (it.tc) {
            st = ensure_b8(it.ds);
            if (st != EPI_OK) return st;
        }
    // graph key: datasets, orders, sizes, path
    std::vector<uint64_t> key;
    key.push_back((uint64_t)path);
    for (auto &it : items) {
        key.push_back(it.ds->id);
        key.push_back((uint64_t)it.k << 32 | (uint64_t)it.top_n);
    }
    char *dev = static_cast<char *>(ctx->batch_dev);
    char *host = static_cast<char *>(ctx->batch_host);
    if (!ctx->batch_exec || key != ctx->batch_key) {
        if (ctx->batch_exec) { cudaGraphExecDestroy(ctx->batch_exec); ctx->batch_exec = nullptr; }
        // descriptor tables, built once per graph
        size_t hp = hoff;
        for (auto &g : groups) {
            const size_t dsz = g.tc ? tc_ds_bytes() : popc_ds_bytes();
            char *hd = host + hp;
            char *hm = hd + dsz * g.items.size();
            int32_t *hc = reinterpret_cast<int32_t *>(hm + 128 * g.items.size());
            for (size_t q = 0; q < g.items.size(); q++) {
                BatchItem &it = items[g.items[q]];
                const DevData d = it.ds->dev();
                uint32_t *thr = reinterpret_cast<uint32_t *>(dev + it.o_thr);
                if (g.tc) {
                    CK(tc_fill_batch_entry(hd + dsz * q, hm + 128 * q, d, it.k, it.ds->b8,
                                           reinterpret_cast<uint64_t *>(dev + it.o_ic), thr, it.total,
                                           dev + g.o_tmap + 128 * q, it.cta_begin, it.cta_count));
                } else {
                    popc_fill_ds(hd + dsz * q, d, 0, it.total, it.cta_begin, it.cta_count, thr);
                }
                for (int c2 = 0; c2 < it.cta_count; c2++) hc[it.cta_begin + c2] = (int32_t)q;
            }
            CK(cudaMemcpyAsync(dev + g.o_desc, hd, dsz * g.items.size(), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(dev + g.o_tmap, hm, 128 * g.items.size(), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(dev + g.o_ctads, hc, (size_t)g.grid * 4, cudaMemcpyHostToDevice, ctx->stream));
            hp = align_up(hp + dsz * g.items.size() + 128 * g.items.size() + (size_t)g.grid * 4, 256);
        }
        CK(cudaStreamSynchronize(ctx->stream));
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        epi_status rs = record_batch(ctx, items, groups, ctx->capture_stream);
        cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (rs != EPI_OK) { if (graph) cudaGraphDestroy(graph); return rs; }
        if (ec != cudaSuccess) return fail(EPI_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ec != cudaSuccess) { ctx->batch_exec = nullptr; return fail(EPI_ECUDA, "graph instantiate: %s", cudaGetErrorString(ec)); }
        ctx->batch_key = key;
    }
    CK(cudaGraphLaunch(ctx->batch_exec, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < n_ds; i++) {
        BatchItem &it = items[i];
        const int32_t code = *reinterpret_cast<int32_t *>(host + it.h_code);
        if (code == EPI_EOVERFLOW) {
            // ties at the pool boundary: this dataset alone, with the retrying search
            st = run_search_sync(it.ds, it.k, it.top_n, it.tc ? EPI_PATH_TC : EPI_PATH_POPC, 0, it.total, outs[i],
                                 counts ? counts[i] : nullptr, &n_outs[i]);
            if (st != EPI_OK) return fail(st, "dataset %d: %s", i, epi_last_error());
            continue;
        }
        if (code != EPI_OK) return fail((epi_status)code, "dataset %d: device status %d", i, code);
        const int n = *reinterpret_cast<int32_t *>(host + it.h_nout);
        memcpy(outs[i], host + it.h_rec, (size_t)n * sizeof(epi_result));
        if (counts && counts[i]) memcpy(counts[i], host + it.h_cnt, (size_t)n * 2 * it.cells * 4);
        n_outs[i] = n;
    }
    return EPI_OK;
}

namespace {

// Device time of one popcount pass over ranks [0, r) with a forced shape, or
// of one whole tensor-core search; < 0 when the shape does not apply.
double time_pass(epi_dataset *ds, int k, bool tc, int R, int tile, int slots, uint64_t r, uint64_t total)
{
    epi_ctx *ctx = ds->ctx;
    SearchPlan p;
    p.k = k; p.top_n = 10; p.pool = initial_pool(10); p.rb = 0; p.re = tc ? total : r; p.total = tc ? total : r;
    p.tc = tc;
    if (tc) {
        p.grid = ctx->num_sms;
    } else {
        p.tile = tile;
        p.slots = slots;
        if (plan_popc(ds, p, R) != EPI_OK || p.tile != tile || p.slots != slots) return -1.0;
    }
    void *dout = nullptr;
    const size_t bytes = 10 * sizeof(epi_result) + 1024;
    if (cudaMallocAsync(&dout, bytes, ctx->stream) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int32_t *status = nullptr;
    double ms = -1.0;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0, ctx->stream);
        const epi_status st = queue_search(ds, p, tc ? EPI_PATH_TC : EPI_PATH_POPC, static_cast<epi_result *>(dout),
                                           nullptr, reinterpret_cast<int32_t *>(static_cast<char *>(dout) + 768), &status);
        cudaEventRecord(e1, ctx->stream);
        if (st != EPI_OK || cudaEventSynchronize(e1) != cudaSuccess) { ms = -1.0; break; }
        float f = 0.0f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = rep ? std::min(ms, (double)f) : (double)f;   // the first run also warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(dout, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return ms;
}

}  // namespace

extern "C" {

epi_status epi_autotune(epi_dataset *ds, int order, int *out)
{
    uint64_t total = 0, re = UINT64_MAX;
    epi_status st = check_search_args(ds, order, 10, EPI_PATH_AUTO, 0, re, total);
    if (st != EPI_OK) return st;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    // probe range: about 16 sub-tiles per resident CTA
    const uint64_t r = std::min<uint64_t>(total, (uint64_t)ctx->num_sms * 8 * 512 * 16);
    std::vector<int> Rs;
    for (int R : {1, 3, 9, 27})
        if (popc_row_group_ok(order, R)) Rs.push_back(R);
    epi_ctx::Tune best;
    best.ms = 1e30;
    for (int R : Rs)
        for (int tile : {128, 256, 512})
            for (int slots : {1, 2, 4, 8}) {
                const double ms = time_pass(ds, order, false, R, tile, slots, r, total);
                if (ms > 0 && ms < best.ms) { best.ms = ms; best.R = R; best.tile = tile; best.slots = slots; }
            }
    if (best.R == 0) return fail(EPI_EUNSUPPORTED, "no popcount launch shape fits this dataset");
    best.path = EPI_PATH_POPC;
    const double popc_full = best.ms * (double)total / (double)r;
    if (tc_applicable(ds, order, 0, total, total)) {
        // the tensor path has no rank ranges: time it whole when that is cheap
        if (popc_full < 4000.0) {
            const double tc_ms = time_pass(ds, order, true, 0, 0, 0, total, total);
            if (tc_ms > 0 && tc_ms < popc_full) best.path = EPI_PATH_TC;
        } else {
            best.path = EPI_PATH_TC;
        }
    }
    ctx->tune[tune_key(order, ds->n, ds->Wt)] = best;
    if (out) { out[0] = best.R; out[1] = best.tile; out[2] = best.slots; out[3] = best.path; }
    return EPI_OK;
}

epi_status epi_tune_save(const epi_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(EPI_EINVAL, "NULL argument");
    FILE *f = fopen(path, "w");
    if (!f) return fail(EPI_EINVAL, "cannot write %s", path);
    fprintf(f, "# libepi autotune cache: key R tile slots path ms\n");
    for (auto &kv : ctx->tune)
        fprintf(f, "%llu %d %d %d %d %.6f\n", (unsigned long long)kv.first, kv.second.R, kv.second.tile,
                kv.second.slots, kv.second.path, kv.second.ms);
    fclose(f);
    return EPI_OK;
}

epi_status epi_tune_load(epi_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(EPI_EINVAL, "NULL argument");
    FILE *f = fopen(path, "r");
    if (!f) return fail(EPI_EINVAL, "cannot read %s", path);
    char line[256];
    int n = 0;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        unsigned long long key = 0;
        epi_ctx::Tune t;
        if (sscanf(line, "%llu %d %d %d %d %lf", &key, &t.R, &t.tile, &t.slots, &t.path, &t.ms) == 6) {
            const int k = (int)(key >> 48);
            if (!popc_row_group_ok(k, t.R) || (t.path != EPI_PATH_POPC && t.path != EPI_PATH_TC)) continue;
            ctx->tune[(uint64_t)key] = t;
            n++;
        }
    }
    fclose(f);
    return EPI_OK;
}

const char *epi_last_error(void) { return g_err.c_str(); }

epi_status epi_search_threshold(epi_dataset *ds, int order, double threshold, int64_t chunk, epi_result *out,
                                int64_t capacity, uint32_t *counts, int64_t *n_found)
{
    uint64_t total = 0, re = UINT64_MAX;
    epi_status st = check_search_args(ds, order, 1, EPI_PATH_POPC, 0, re, total);
    if (st != EPI_OK) return st;
    if (!n_found || capacity < 0 || (capacity > 0 && !out) || !std::isfinite(threshold) || chunk < 0)
        return fail(EPI_EINVAL, "epi_search_threshold: bad argument");
    *n_found = 0;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t sm = ctx->stream;
    const DevData d = ds->dev();
    const int cells = pow3i(order);
    // FP32 screen: a combination with MI >= threshold scores at least
    // threshold (1 - bound) in single precision (the bound covers the
    // roundings of the 2 * 3^k terms); the FP64 value decides
    const float thr32 = threshold > 0.0 ? (float)(threshold * (1.0 - 2.0 * f32_rel_bound(order, ds->m))) : -INFINITY;
    const uint64_t ch = chunk > 0 ? std::min<uint64_t>((uint64_t)chunk, total) : std::min<uint64_t>(total, 1ull << 28);
    const int64_t slice = std::max<int64_t>(1, std::min<int64_t>(1 << 20, ((int64_t)256 << 20) / (8 * cells)));
    float *scores = nullptr;
    unsigned long long *n_dev = nullptr;
    uint64_t *cand = nullptr;
    uint32_t *combs = nullptr, *tabs = nullptr;
    float *f32 = nullptr;
    double *f64 = nullptr;
    void *dout = nullptr;
    uint64_t cand_cap = std::min<uint64_t>(ch, 1ull << 20);
    struct Found {
        uint64_t rank;
        double mi;
        float mi32;
        std::vector<uint32_t> snp, tab;
    };
    std::vector<Found> found;
    int64_t n_qual = 0;
    auto better = [](const Found &a, const Found &b) { return a.mi > b.mi || (a.mi == b.mi && a.rank < b.rank); };
    // only the best `capacity` are kept (pruned whenever the list doubles)
    auto prune = [&]() {
        if ((int64_t)found.size() <= capacity) return;
        std::nth_element(found.begin(), found.begin() + capacity, found.end(), better);
        found.resize((size_t)capacity);
    };
    auto cleanup = [&]() {
        for (void *q : {(void *)scores, (void *)n_dev, (void *)cand, (void *)combs, (void *)tabs, (void *)f32,
                        (void *)f64, dout})
            if (q) cudaFreeAsync(q, sm);
        cudaStreamSynchronize(sm);
    };
#define TCK(call)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            cleanup();                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? EPI_ENOMEM : EPI_ECUDA,    \
                        "epi_search_threshold: %s", cudaGetErrorString(e_));         \
        }                                                                            \
    } while (0)
    TCK(cudaMallocAsync((void **)&scores, (size_t)ch * 4, sm));
    TCK(cudaMallocAsync((void **)&n_dev, 8, sm));
    TCK(cudaMallocAsync((void **)&cand, (size_t)cand_cap * 8, sm));
    TCK(cudaMallocAsync((void **)&combs, (size_t)slice * order * 4, sm));
    TCK(cudaMallocAsync((void **)&tabs, (size_t)slice * 2 * cells * 4, sm));
    TCK(cudaMallocAsync((void **)&f32, (size_t)slice * 4, sm));
    TCK(cudaMallocAsync((void **)&f64, (size_t)slice * 8, sm));
    TCK(cudaMallocAsync(&dout, 1024, sm));
    std::vector<uint32_t> hc, ht;
    std::vector<double> h64;
    std::vector<float> h32;
    std::vector<uint64_t> hr;
    for (uint64_t rb = 0; rb < total; rb += ch) {
        // every score of ranks [rb, rb + ch): the popcount path
        SearchPlan p;
        p.k = order; p.top_n = 1; p.pool = initial_pool(1); p.rb = rb; p.re = std::min(total, rb + ch); p.total = total;
        p.all_scores = scores;
        st = plan_popc(ds, p);
        if (st != EPI_OK) { cleanup(); return st; }
        int32_t *status = nullptr;
        st = queue_search(ds, p, EPI_PATH_POPC, static_cast<epi_result *>(dout), nullptr,
                          reinterpret_cast<int32_t *>(static_cast<char *>(dout) + 512), &status);
        if (st != EPI_OK) { cleanup(); return st; }
        const int64_t cnt = (int64_t)(p.re - p.rb);
        // the candidates of the FP32 screen
        unsigned long long nc = 0;
        for (;;) {
            TCK(cudaMemsetAsync(n_dev, 0, 8, sm));
            TCK(launch_select_ge(scores, cnt, thr32, rb, cand, cand_cap, n_dev, ctx->num_sms, sm));
            TCK(cudaMemcpyAsync(&nc, n_dev, 8, cudaMemcpyDeviceToHost, sm));
            TCK(cudaStreamSynchronize(sm));
            ctx->launches += 2;
            if (nc <= cand_cap) break;
            cudaFreeAsync(cand, sm);
            cand = nullptr;
            cand_cap = nc;
            TCK(cudaMallocAsync((void **)&cand, (size_t)cand_cap * 8, sm));
        }
        // exact FP64 scores of the candidates, in slices
        for (int64_t off = 0; off < (int64_t)nc; off += slice) {
            const int64_t c = std::min<int64_t>(slice, (int64_t)nc - off);
            TCK(launch_unrank(d, order, cand + off, c, combs, sm));
            TCK(launch_tables(d, order, combs, c, tabs, ctx->num_sms, sm));
            TCK(launch_score_tables(d, order, tabs, c, f32, f64, ctx->num_sms, sm));
            ctx->launches += 3;
            hr.resize(c); hc.resize((size_t)c * order); h64.resize(c); h32.resize(c);
            TCK(cudaMemcpyAsync(hr.data(), cand + off, (size_t)c * 8, cudaMemcpyDeviceToHost, sm));
            TCK(cudaMemcpyAsync(hc.data(), combs, (size_t)c * order * 4, cudaMemcpyDeviceToHost, sm));
            TCK(cudaMemcpyAsync(h64.data(), f64, (size_t)c * 8, cudaMemcpyDeviceToHost, sm));
            TCK(cudaMemcpyAsync(h32.data(), f32, (size_t)c * 4, cudaMemcpyDeviceToHost, sm));
            if (counts) {
                ht.resize((size_t)c * 2 * cells);
                TCK(cudaMemcpyAsync(ht.data(), tabs, ht.size() * 4, cudaMemcpyDeviceToHost, sm));
            }
            TCK(cudaStreamSynchronize(sm));
            for (int64_t i = 0; i < c; i++) {
                if (!(h64[i] >= threshold)) continue;
                n_qual++;
                if (capacity == 0) continue;
                Found f;
                f.rank = hr[i];
                f.mi = h64[i];
                f.mi32 = h32[i];
                f.snp.assign(hc.begin() + i * order, hc.begin() + (i + 1) * order);
                if (counts) f.tab.assign(ht.begin() + i * 2 * cells, ht.begin() + (i + 1) * 2 * cells);
                found.push_back(std::move(f));
                if ((int64_t)found.size() >= 2 * capacity + 1024) prune();
            }
        }
    }
#undef TCK
    cleanup();
    prune();
    std::sort(found.begin(), found.end(), better);
    *n_found = n_qual;
    const int64_t n_out = std::min<int64_t>(capacity, (int64_t)found.size());
    for (int64_t q = 0; q < n_out; q++) {
        epi_result r;
        std::memset(&r, 0, sizeof(r));
        for (int t = 0; t < order; t++) r.snp[t] = found[q].snp[t];
        r.mi = found[q].mi;
        r.mi_f32 = found[q].mi32;
        r.order = order;
        r.rank = found[q].rank;
        out[q] = r;
        if (counts) std::memcpy(counts + (size_t)q * 2 * cells, found[q].tab.data(), (size_t)2 * cells * 4);
    }
    return EPI_OK;
}

epi_status epi_score_all(epi_dataset *ds, int order, float *out_dev)
{
    uint64_t total = 0, re = UINT64_MAX;
    epi_status st = check_search_args(ds, order, 1, EPI_PATH_POPC, 0, re, total);
    if (st != EPI_OK) return st;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    if (!out_dev || !is_device_ptr(out_dev, ctx->device))
        return fail(EPI_EINVAL, "epi_score_all: out must be device memory of device %d", ctx->device);
    SearchPlan p;
    p.k = order; p.top_n = 1; p.pool = initial_pool(1); p.rb = 0; p.re = total; p.total = total;
    p.all_scores = out_dev;
    st = plan_popc(ds, p);
    if (st != EPI_OK) return st;
    void *dout = nullptr;
    CK(cudaMallocAsync(&dout, 1024, ctx->stream));
    int32_t *status = nullptr;
    st = queue_search(ds, p, EPI_PATH_POPC, static_cast<epi_result *>(dout), nullptr,
                      reinterpret_cast<int32_t *>(static_cast<char *>(dout) + 512), &status);
    cudaFreeAsync(dout, ctx->stream);
    if (st != EPI_OK) return st;
    CK(cudaStreamSynchronize(ctx->stream));
    return EPI_OK;
}

epi_status epi_unrank(epi_dataset *ds, int order, const uint64_t *ranks, int64_t count, uint32_t *combs)
{
    if (!ds || !ranks || !combs || count < 0) return fail(EPI_EINVAL, "epi_unrank: bad argument");
    if (order < 1 || order > EPI_MAX_ORDER || order > ds->n) return fail(EPI_EINVAL, "epi_unrank: bad order");
    if (count == 0) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    CK(launch_unrank(ds->dev(), order, ranks, count, combs, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_features5(epi_dataset *ds, const float *s1, const float *s2, const float *s3, const float *s4,
                         const uint32_t *combs, int64_t count, float *X)
{
    if (!ds || !s1 || !s2 || !s3 || !combs || !X || count < 0) return fail(EPI_EINVAL, "epi_features5: bad argument");
    if (ds->n < 5) return fail(EPI_EINVAL, "epi_features5: needs at least 5 SNPs");
    if (count == 0) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    CK(launch_features5(ds->dev(), s1, s2, s3, s4, combs, count, X, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_candidates5(epi_dataset *ds, const uint32_t *triples, int64_t n_triples, int64_t first, int64_t count,
                           uint32_t *combs, const float *s3, uint8_t *keep)
{
    if ((s3 == nullptr) != (keep == nullptr)) return fail(EPI_EINVAL, "epi_candidates5: give both s3 and keep, or neither");
    if (!ds || !triples || !combs || first < 0 || count < 0) return fail(EPI_EINVAL, "epi_candidates5: bad argument");
    const int64_t rest = ds->n - 3;
    if (rest < 2) return fail(EPI_EINVAL, "epi_candidates5: needs at least 5 SNPs");
    const int64_t per = rest * (rest - 1) / 2;
    if (first + count > n_triples * per) return fail(EPI_EINVAL, "epi_candidates5: range beyond the candidate space");
    if (count == 0) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    CK(launch_candidates5(ds->dev(), triples, first, count, combs, s3, keep, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_score5(epi_dataset *ds, const uint32_t *combs, int64_t count, float *out)
{
    if (!ds || !combs || !out || count < 0) return fail(EPI_EINVAL, "epi_score5: bad argument");
    if (ds->n < 5) return fail(EPI_EINVAL, "epi_score5: needs at least 5 SNPs");
    if (count == 0) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!is_device_ptr(combs, ctx->device) || !is_device_ptr(out, ctx->device))
        return fail(EPI_EINVAL, "epi_score5: combs and out must be device memory of device %d", ctx->device);
    CK(launch_score5_f32(ds->dev(), combs, count, out, ctx->num_sms, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_lookup(epi_dataset *ds, int order, const float *table, const uint32_t *combs, int64_t count, float *out)
{
    if (!ds || !table || !combs || !out || count < 0) return fail(EPI_EINVAL, "epi_lookup: bad argument");
    if (order < 1 || order > EPI_MAX_ORDER || order > ds->n) return fail(EPI_EINVAL, "epi_lookup: bad order");
    if (count == 0) return EPI_OK;
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    CK(launch_lookup(ds->dev(), order, table, combs, count, out, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_topk(epi_ctx *ctx, const float *scores, const uint8_t *keep, int64_t count, int k, float *out_scores,
                    uint64_t *out_index, int32_t *n_out)
{
    if (!ctx || !scores || !out_scores || !out_index || !n_out || count < 0) return fail(EPI_EINVAL, "epi_topk: bad argument");
    if (k < 1 || k > 4096) return fail(EPI_EINVAL, "epi_topk: k outside 1..4096");
    DeviceGuard g(ctx->device);
    epi_status st = ensure_scratch(ctx, topk_scratch_bytes(k));
    if (st != EPI_OK) return st;
    CK(launch_topk(scores, keep, count, k, ctx->scratch, true, out_scores, out_index, n_out, ctx->num_sms, ctx->stream));
    ctx->launches += 14;
    return EPI_OK;
}

}  // extern "C"

cudaStream_t epi_ctx_stream(const epi_ctx *ctx) { return ctx->stream; }
int epi_ctx_device(const epi_ctx *ctx) { return ctx->device; }
int epi_ctx_num_sms(const epi_ctx *ctx) { return ctx->num_sms; }
void epi_ctx_count_launches(epi_ctx *ctx, int n) { ctx->launches += (uint64_t)n; }
epi_ctx *epi_dataset_ctx(const epi_dataset *ds) { return ds->ctx; }
epi::DevData epi_dataset_dev(const epi_dataset *ds) { return ds->dev(); }

// The dataset's exhaustive single-precision scores of order k (1..4), computed
// on first use and kept until the dataset is destroyed.
epi_status epi_dataset_lower_scores(epi_dataset *ds, int k, const float **out)
{
    if (k < 1 || k > 4 || k > ds->n) return fail(EPI_EINVAL, "lower scores: order %d outside 1..min(4, n)", k);
    if (!ds->lower[k]) {
        DeviceGuard g(ds->ctx->device);
        float *t = nullptr;
        CK(cudaMalloc(&t, (size_t)host_binom(ds->n, k) * sizeof(float)));
        const epi_status st = epi_score_all(ds, k, t);
        if (st != EPI_OK) {
            cudaFree(t);
            return st;
        }
        ds->lower[k] = t;
    }
    *out = ds->lower[k];
    return EPI_OK;
}

extern "C" {

epi_status epi_create(int device, void *cuda_stream, epi_ctx **out)
{
    if (!out) return fail(EPI_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    CK(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(EPI_EINVAL, "device %d outside 0..%d", device, count - 1);
    DeviceGuard g(device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", device);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(EPI_EUNSUPPORTED, "device %d is sm_%d%d; the library targets sm_103a", device,
                                     prop.major, prop.minor);
    epi_ctx *c = new epi_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *out = c;
    return EPI_OK;
}

static void free_ctx(epi_ctx *ctx)
{
    DeviceGuard g(ctx->device);
    if (ctx->scratch) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->scratch);
    }
    for (auto &pr : ctx->prof_events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    if (ctx->waits_dev) cudaFree(ctx->waits_dev);
    if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
    if (ctx->batch_dev) cudaFree(ctx->batch_dev);
    if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
}

void epi_destroy(epi_ctx *ctx)
{
    if (!ctx) return;
    // a context outlives its datasets: the last epi_dataset_destroy frees it
    ctx->destroy_requested = true;
    if (ctx->live_datasets == 0) free_ctx(ctx);
}

epi_status epi_dataset_create(epi_ctx *ctx, const uint8_t *geno, const uint8_t *pheno, int64_t n_snps,
                              int64_t n_samples, int inputs_on_device, epi_dataset **out)
{
    if (!ctx || !geno || !pheno || !out) return fail(EPI_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_snps < 1 || n_samples < 1) return fail(EPI_EINVAL, "need at least one SNP and one sample");
    if (n_samples > (1 << 23) - 1) return fail(EPI_EINVAL, "n_samples %lld above 2^23-1", (long long)n_samples);
    if (n_snps > (1 << 24)) return fail(EPI_EINVAL, "n_snps %lld above 2^24", (long long)n_snps);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t st = ctx->stream;
    const int64_t n = n_snps, m = n_samples;
    uint8_t *dgeno = nullptr, *dpheno = nullptr, *tmp = nullptr;
    if (inputs_on_device) {
        if (!is_device_ptr(geno, ctx->device) || !is_device_ptr(pheno, ctx->device))
            return fail(EPI_EINVAL, "inputs_on_device set but geno/pheno are not device memory of device %d",
                        ctx->device);
        dgeno = const_cast<uint8_t *>(geno);
        dpheno = const_cast<uint8_t *>(pheno);
    } else {
        CK(ctx_malloc_async(ctx, (void **)&tmp, (size_t)(n * m + m), st));
        dgeno = tmp;
        dpheno = tmp + n * m;
        CK(cudaMemcpyAsync(dgeno, geno, (size_t)(n * m), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dpheno, pheno, (size_t)m, cudaMemcpyHostToDevice, st));
    }
    void *work = nullptr;
    const size_t work_bytes = (size_t)m * 8 + 64;
    {
        const cudaError_t ew = ctx_malloc_async(ctx, &work, work_bytes, st);
        if (ew != cudaSuccess) {
            if (tmp) cudaFreeAsync(tmp, st);
            cudaStreamSynchronize(st);
            return fail(ew == cudaErrorMemoryAllocation ? EPI_ENOMEM : EPI_ECUDA, "dataset work buffer: %s",
                        cudaGetErrorString(ew));
        }
    }
    int32_t *case_idx = static_cast<int32_t *>(work);
    int32_t *ctrl_idx = case_idx + m;
    // 2 m int32 entries end on an 8-byte boundary
    int64_t *dm1 = reinterpret_cast<int64_t *>(case_idx + 2 * m);
    int32_t *dstatus = reinterpret_cast<int32_t *>(dm1 + 1);
    CK(cudaMemsetAsync(dstatus, 0, 4, st));
    launch_scan_pheno(dpheno, m, case_idx, ctrl_idx, dm1, dstatus, st);
    CK(cudaGetLastError());
    int64_t m1 = 0;
    int32_t hstatus = 0;
    CK(cudaMemcpyAsync(&m1, dm1, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hstatus, dstatus, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    epi_status ret = EPI_OK;
    epi_dataset *ds = nullptr;
    if (hstatus & ST_BAD_PHENO) {
        ret = fail(EPI_EINVAL, "phenotype values must be 0 or 1");
    } else {
        ds = new epi_dataset();
        ds->ctx = ctx;
        ds->id = ctx->next_dataset_id++;
        ds->n = n; ds->m = m; ds->m1 = m1; ds->m0 = m - m1;
        ds->W1 = (int32_t)(((m1 + 127) / 128) * 4);
        ds->W0 = (int32_t)(((m - m1 + 127) / 128) * 4);
        ds->Wt = ds->W1 + ds->W0;
        cudaError_t e1 = ctx_malloc(ctx, (void **)&ds->masks, (size_t)n * 3 * ds->Wt * 4);
        cudaError_t e2 = ctx_malloc(ctx, (void **)&ds->binom, (size_t)9 * (n + 1) * 8);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            ret = fail(EPI_ENOMEM, "dataset allocation failed");
        } else {
            launch_pack_masks(dgeno, n, m, case_idx, ctrl_idx, m1, ds->W1, ds->Wt, ds->masks, dstatus, ctx->num_sms, st);
            launch_binom(n, ds->binom, ctx->num_sms, st);
            ctx->launches += 3;
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, dstatus, 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) ret = fail(EPI_ECUDA, "packing failed: %s", cudaGetErrorString(e));
            else if (hstatus & ST_BAD_GENO) ret = fail(EPI_EINVAL, "genotype values must be 0, 1 or 2");
        }
    }
    cudaFreeAsync(work, st);
    if (tmp) cudaFreeAsync(tmp, st);
    cudaStreamSynchronize(st);
    if (ret != EPI_OK) {
        if (ds) { cudaFree(ds->masks); cudaFree(ds->binom); delete ds; }
        return ret;
    }
    ctx->live_datasets++;
    *out = ds;
    return EPI_OK;
}

void epi_dataset_destroy(epi_dataset *ds)
{
    if (!ds) return;
    epi_ctx *ctx = ds->ctx;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ds->masks);
        cudaFree(ds->binom);
        if (ds->b8) cudaFree(ds->b8);
        if (ds->b8c) cudaFree(ds->b8c);
        for (float *t : ds->lower)
            if (t) cudaFree(t);
    }
    delete ds;
    ctx->live_datasets--;
    if (ctx->destroy_requested && ctx->live_datasets == 0) free_ctx(ctx);
}

epi_status epi_dataset_info(const epi_dataset *ds, int64_t *n_snps, int64_t *n_samples, int64_t *n_cases,
                            int64_t *n_controls)
{
    if (!ds) return fail(EPI_EINVAL, "dataset is NULL");
    if (n_snps) *n_snps = ds->n;
    if (n_samples) *n_samples = ds->m;
    if (n_cases) *n_cases = ds->m1;
    if (n_controls) *n_controls = ds->m0;
    return EPI_OK;
}

epi_status epi_search(epi_dataset *ds, int order, int top_n, int path, epi_result *out, uint32_t *counts, int *n_out)
{
    return run_search_sync(ds, order, top_n, path, 0, UINT64_MAX, out, counts, n_out);
}

epi_status epi_search_range(epi_dataset *ds, int order, int top_n, int path, uint64_t rank_begin, uint64_t rank_end,
                            epi_result *out, uint32_t *counts, int *n_out)
{
    return run_search_sync(ds, order, top_n, path, rank_begin, rank_end, out, counts, n_out);
}

epi_status epi_search_async(epi_dataset *ds, int order, int top_n, int path, epi_result *out_dev,
                            uint32_t *counts_dev, int32_t *n_out_dev, int32_t *status_dev)
{
    uint64_t total = 0, re = UINT64_MAX;
    epi_status st = check_search_args(ds, order, top_n, path, 0, re, total);
    if (st != EPI_OK) return st;
    if (!out_dev || !n_out_dev || !status_dev) return fail(EPI_EINVAL, "NULL output pointer");
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    if (!is_device_ptr(out_dev, ctx->device) || !is_device_ptr(n_out_dev, ctx->device) ||
        !is_device_ptr(status_dev, ctx->device) || (counts_dev && !is_device_ptr(counts_dev, ctx->device)))
        return fail(EPI_EINVAL, "epi_search_async outputs must be device memory of device %d", ctx->device);
    SearchPlan p;
    p.k = order; p.top_n = top_n; p.pool = initial_pool(top_n); p.rb = 0; p.re = re; p.total = total;
    st = make_plan(ds, p, path);
    if (st != EPI_OK) return st;
    int32_t *status = nullptr;
    st = queue_search(ds, p, path, out_dev, counts_dev, n_out_dev, &status);
    if (st != EPI_OK) return st;
    // device status bits to an epi_status code
    CK(launch_publish_status(status, status_dev, ctx->stream));
    ctx->launches += 1;
    return EPI_OK;
}

epi_status epi_tables(epi_dataset *ds, int order, const uint32_t *combs, int64_t count, uint32_t *out)
{
    if (!ds) return fail(EPI_EINVAL, "dataset is NULL");
    if (order < 1 || order > EPI_MAX_ORDER) return fail(EPI_EINVAL, "order %d outside 1..%d", order, EPI_MAX_ORDER);
    if (count < 0) return fail(EPI_EINVAL, "negative count");
    if (count == 0) return EPI_OK;
    if (!combs || !out) return fail(EPI_EINVAL, "NULL argument");
    for (int64_t c = 0; c < count; c++)
        for (int t = 0; t < order; t++) {
            const uint32_t v = combs[c * order + t];
            if (v >= (uint64_t)ds->n || (t && v <= combs[c * order + t - 1]))
                return fail(EPI_EINVAL, "combination %lld is not strictly increasing within 0..%lld", (long long)c,
                            (long long)ds->n - 1);
        }
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    const size_t cells = (size_t)pow3i(order);
    const size_t in_b = (size_t)count * order * 4, out_b = (size_t)count * 2 * cells * 4;
    void *buf = nullptr;
    CK(cudaMallocAsync(&buf, in_b + out_b + 256, ctx->stream));
    uint32_t *dc = static_cast<uint32_t *>(buf);
    uint32_t *dout = reinterpret_cast<uint32_t *>(static_cast<char *>(buf) + ((in_b + 255) & ~(size_t)255));
    cudaError_t e = cudaMemcpyAsync(dc, combs, in_b, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_tables(ds->dev(), order, dc, count, dout, ctx->num_sms, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, out_b, cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(buf, ctx->stream);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(EPI_ECUDA, "tables: %s", cudaGetErrorString(e));
    return EPI_OK;
}

epi_status epi_score_tables(epi_dataset *ds, int order, const uint32_t *tables, int64_t count, float *mi_f32,
                            double *mi_f64)
{
    if (!ds) return fail(EPI_EINVAL, "dataset is NULL");
    if (order < 1 || order > EPI_MAX_ORDER) return fail(EPI_EINVAL, "order %d outside 1..%d", order, EPI_MAX_ORDER);
    if (count < 0) return fail(EPI_EINVAL, "negative count");
    if (count == 0) return EPI_OK;
    if (!tables) return fail(EPI_EINVAL, "NULL tables");
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    const size_t cells = (size_t)pow3i(order);
    const size_t in_b = (size_t)count * 2 * cells * 4;
    void *buf = nullptr;
    CK(cudaMallocAsync(&buf, in_b + (size_t)count * 12 + 512, ctx->stream));
    uint32_t *dt = static_cast<uint32_t *>(buf);
    char *p = static_cast<char *>(buf) + ((in_b + 255) & ~(size_t)255);
    double *d64 = reinterpret_cast<double *>(p);
    float *d32 = reinterpret_cast<float *>(p + (((size_t)count * 8 + 255) & ~(size_t)255));
    cudaError_t e = cudaMemcpyAsync(dt, tables, in_b, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_score_tables(ds->dev(), order, dt, count, d32, d64, ctx->num_sms, ctx->stream);
    if (e == cudaSuccess && mi_f32) e = cudaMemcpyAsync(mi_f32, d32, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && mi_f64) e = cudaMemcpyAsync(mi_f64, d64, (size_t)count * 8, cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(buf, ctx->stream);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(EPI_ECUDA, "score_tables: %s", cudaGetErrorString(e));
    return EPI_OK;
}

uint64_t epi_kernel_launches(const epi_ctx *ctx) { return ctx ? ctx->launches : 0; }

epi_status epi_debug_counts(epi_dataset *ds, int order, uint32_t *out)
{
    uint64_t total = 0, re = UINT64_MAX;
    epi_status st = check_search_args(ds, order, 1, EPI_PATH_TC, 0, re, total);
    if (st != EPI_OK) return st;
    if (!out) return fail(EPI_EINVAL, "out is NULL");
    if (!tc_applicable(ds, order, 0, total, total))
        return fail(EPI_EUNSUPPORTED, "the tensor-core path does not apply to this dataset and order");
    const size_t cells = (size_t)pow3i(order);
    const size_t bytes = (size_t)total * 2 * cells * 4;
    if (bytes > ((size_t)1 << 31)) return fail(EPI_EINVAL, "debug table dump limited to 2 GiB");
    epi_ctx *ctx = ds->ctx;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    SearchPlan p;
    p.k = order; p.top_n = 1; p.pool = initial_pool(1); p.rb = 0; p.re = total; p.total = total;
    st = make_plan(ds, p, EPI_PATH_TC);
    if (st != EPI_OK) return st;
    void *buf = nullptr;
    CK(cudaMallocAsync(&buf, bytes + sizeof(epi_result) + 512, ctx->stream));
    uint32_t *dump = static_cast<uint32_t *>(buf);
    epi_result *rec = reinterpret_cast<epi_result *>(static_cast<char *>(buf) + ((bytes + 255) & ~(size_t)255));
    int32_t *nout = reinterpret_cast<int32_t *>(rec + 1);
    int32_t *status = nullptr;
    cudaError_t e = cudaMemsetAsync(dump, 0xff, bytes, ctx->stream);
    if (e != cudaSuccess) { cudaFreeAsync(buf, ctx->stream); return fail(EPI_ECUDA, "%s", cudaGetErrorString(e)); }
    st = queue_search(ds, p, EPI_PATH_TC, rec, nullptr, nout, &status, dump);
    if (st == EPI_OK) {
        int32_t hs = 0;
        e = cudaMemcpyAsync(out, dump, bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(EPI_ECUDA, "%s", cudaGetErrorString(e));
        else if (hs & ST_TIMEOUT) st = fail(EPI_ETIMEOUT, "device wait expired");
    }
    cudaFreeAsync(buf, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return st;
}

epi_status epi_count_variant(epi_dataset *ds, int order, int variant, uint32_t *tables, uint64_t *checksum,
                             double *ms)
{
    if (!ds || !checksum) return fail(EPI_EINVAL, "NULL argument");
    if (order < 2 || order > 4) return fail(EPI_EINVAL, "order %d outside 2..4", order);
    if (variant < 0 || variant > 2) return fail(EPI_EINVAL, "variant %d outside 0..2", variant);
    if (order > ds->n) return fail(EPI_EINVAL, "order %d exceeds the %lld SNPs", order, (long long)ds->n);
    epi_ctx *ctx = ds->ctx;
    const uint64_t total = host_binom(ds->n, order);
    const size_t cells = (size_t)pow3i(order);
    const size_t bytes = tables ? (size_t)total * 2 * cells * 4 : 0;
    if (tables && bytes > ((size_t)1 << 31)) return fail(EPI_EINVAL, "table dump limited to 2 GiB");
    if (count_variant_smem_bytes(order, ds->Wt) > ctx->smem_optin)
        return fail(EPI_EUNSUPPORTED, "one prefix table does not fit in shared memory");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    void *buf = nullptr;
    CK(ctx_malloc_async(ctx, &buf, bytes + 256, ctx->stream));
    unsigned long long *sum = static_cast<unsigned long long *>(buf);
    uint32_t *dtab = tables ? reinterpret_cast<uint32_t *>(static_cast<char *>(buf) + 256) : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float t = 0.0f;
    unsigned long long hsum = 0;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, 8, ctx->stream);
    if (e == cudaSuccess && dtab) e = cudaMemsetAsync(dtab, 0xff, bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess)
        e = launch_count_variant(ds->dev(), order, variant, total, dtab, sum, ctx->num_sms * 8, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hsum, sum, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && dtab) e = cudaMemcpyAsync(tables, dtab, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(EPI_ECUDA, "%s", cudaGetErrorString(e));
    ctx->launches += 1;
    *checksum = hsum;
    if (ms) *ms = (double)t;
    return EPI_OK;
}

epi_status epi_set_wait_limit(epi_ctx *ctx, uint64_t limit_ns)
{
    if (!ctx) return fail(EPI_EINVAL, "context is NULL");
    ctx->wait_limit_ns = limit_ns;
    return EPI_OK;
}

epi_status epi_inject_alloc_failure(epi_ctx *ctx, int64_t after)
{
    if (!ctx) return fail(EPI_EINVAL, "context is NULL");
    ctx->fail_alloc_in = after < 0 ? -1 : after;
    return EPI_OK;
}

epi_status epi_set_tc_variant(epi_ctx *ctx, int variant)
{
    if (!ctx) return fail(EPI_EINVAL, "context is NULL");
    if (variant != EPI_TC_AUTO && variant != EPI_TC_SEPARATE) return fail(EPI_EINVAL, "variant %d unknown", variant);
    ctx->tc_combined = variant == EPI_TC_AUTO;
    return EPI_OK;
}

epi_status epi_tc_rate(epi_ctx *ctx, int shape, int64_t stages, double *out)
{
    if (!ctx || !out) return fail(EPI_EINVAL, "NULL argument");
    if (shape != 0 && shape != 1) return fail(EPI_EINVAL, "shape %d unknown", shape);
    if (stages < 32 || stages > ((int64_t)1 << 32)) return fail(EPI_EINVAL, "stages outside 32..2^32");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EPI_ECUDA, "cannot select device %d", ctx->device);
    const int grid = ctx->num_sms;
    void *buf = nullptr;
    CK(cudaMallocAsync(&buf, (size_t)grid * 8 + 256, ctx->stream));
    unsigned long long *cycles = static_cast<unsigned long long *>(buf);
    int32_t *status = reinterpret_cast<int32_t *>(static_cast<char *>(buf) + (size_t)grid * 8);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<unsigned long long> cyc((size_t)grid);
    int32_t hs = 0;
    float ms = 0.0f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, ctx->stream);
    // a short warm-up launch, then the timed one
    if (e == cudaSuccess) e = launch_mma_rate(shape, 32, cycles, status, grid, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess) e = launch_mma_rate(shape, stages, cycles, status, grid, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cyc.data(), cycles, (size_t)grid * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(EPI_ECUDA, "%s", cudaGetErrorString(e));
    if (hs & ST_TIMEOUT) return fail(EPI_ETIMEOUT, "device wait expired");
    ctx->launches += 2;
    const double macs_per_sm = (double)stages * 4.0 * 128.0 * (shape ? 256.0 : 128.0) * 32.0;
    double mean_cyc = 0.0;
    for (unsigned long long c : cyc) mean_cyc += (double)c;
    mean_cyc /= (double)grid;
    out[0] = 2.0 * macs_per_sm * grid / ((double)ms * 1e-3) / 1e12;
    out[1] = macs_per_sm / mean_cyc;
    out[2] = (double)ms;
    out[3] = mean_cyc / ((double)ms * 1e3);
    return EPI_OK;
}

epi_status epi_profile_begin(epi_ctx *ctx)
{
    if (!ctx) return fail(EPI_EINVAL, "context is NULL");
    DeviceGuard g(ctx->device);
    for (auto &pr : ctx->prof_events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    ctx->prof_events.clear();
    ctx->profiling = true;
    ctx->waits_grid = 0;
    return EPI_OK;
}

epi_status epi_profile_waits(epi_ctx *ctx, double *out)
{
    if (!ctx || !out) return fail(EPI_EINVAL, "NULL argument");
    for (int i = 0; i < kTcWaitSlots; i++) out[i] = 0.0;
    if (!ctx->waits_dev || ctx->waits_grid <= 0) return EPI_OK;
    DeviceGuard g(ctx->device);
    std::vector<unsigned long long> h((size_t)ctx->waits_grid * kTcWaitSlots);
    CK(cudaMemcpyAsync(h.data(), ctx->waits_dev, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < ctx->waits_grid; b++)
        for (int i = 0; i < kTcWaitSlots; i++) out[i] += (double)h[(size_t)b * kTcWaitSlots + i] / ctx->waits_grid;
    return EPI_OK;
}

epi_status epi_profile_end(epi_ctx *ctx, double *kernel_ms, int64_t *launches)
{
    if (!ctx || !kernel_ms || !launches) return fail(EPI_EINVAL, "NULL argument");
    DeviceGuard g(ctx->device);
    double total = 0.0;
    epi_status st = EPI_OK;
    for (auto &pr : ctx->prof_events) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess && st == EPI_OK) st = fail(EPI_ECUDA, "profile events: %s", cudaGetErrorString(e));
        total += ms;
    }
    *kernel_ms = total;
    *launches = (int64_t)ctx->prof_events.size();
    for (auto &pr : ctx->prof_events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    ctx->prof_events.clear();
    ctx->profiling = false;
    return st;
}

}  // extern "C"
