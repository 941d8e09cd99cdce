// Learned order-5 proposer: the pipelines around the network.
//
// Search: the exhaustive order-1..3 scores (the popcount path; with the
// 30-feature set also order 4) give the features; the best T triples by
// order-3 score are expanded by every pair of other SNPs; each distinct expansion is ranked by the network (or by
// the network-free heuristic), the best R are recounted and scored exactly
// (tables and FP64 MI of Eq. 1-3), and the best top_n of those are returned.
//
// Training: the same expansions of training datasets are labelled with their
// exact order-5 MI (every row's table counted and scored, Section 2.2 and
// Eq. 1-3) and the network is fitted to ln(MI + 1e-7), standardised,
// by AdamW on mini-batches drawn on the device; part of every batch comes from
// each dataset's best-labelled rows, where the ranking matters.
//
// Every step runs in the library's kernels; the host only sequences them,
// sorts the final R exact scores and keeps the index lists of the rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "epi_host.h"
#include "epi_internal.cuh"

namespace epi {

void set_last_error(const char *msg);

namespace prop {

__global__ void count_kernel(const uint8_t *__restrict__ keep, int64_t count, unsigned long long *out)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        c += keep[i];
    for (int off = 16; off; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// t[i] = ln(max(s, 0) + 1e-7): the training label of an exact order-5 score
__global__ void log_label_kernel(float *t, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = logf(fmaxf(t[i], 0.0f) + 1e-7f);
}

// mean and standard deviation of column f of X [rows][cols] (one block per
// column, FP64 sums in a fixed order)
__global__ void __launch_bounds__(256) moments_kernel(const float *__restrict__ X, int64_t rows, int cols,
                                                      double *__restrict__ out)
{
    const int f = blockIdx.x;
    double s = 0.0, q = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        const double v = X[r * cols + f];
        s += v;
        q += v * v;
    }
    __shared__ double ps[256], pq[256];
    ps[threadIdx.x] = s;
    pq[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if ((int)threadIdx.x < w) { ps[threadIdx.x] += ps[threadIdx.x + w]; pq[threadIdx.x] += pq[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = ps[0] / (double)rows;
        const double var = fmax(pq[0] / (double)rows - mean * mean, 0.0);
        out[2 * f] = mean;
        out[2 * f + 1] = sqrt(var);
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// t[tail[i]] = 1 for the listed rows (the membership labels start at 0)
__global__ void mark_kernel(float *t, const uint64_t *tail, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        t[tail[i]] = 1.0f;
}

// One mini-batch: row i draws a SplitMix64 value of (seed, step, i) and takes
// that position of the tail list (i < n_tail_rows) or of the kept list; the
// label is (t - t_mean) * t_inv_sd.
__global__ void gather_batch_kernel(const float *__restrict__ X, const float *__restrict__ t, int cols,
                                    const uint64_t *__restrict__ kept, uint64_t n_kept, const uint64_t *__restrict__ tail,
                                    uint64_t n_tail, int batch, int n_tail_rows, uint64_t seed, uint64_t step,
                                    float t_mean, float t_inv_sd, float *__restrict__ Xb, float *__restrict__ tb)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        const uint64_t h = mix64(seed + 0x9E3779B97F4A7C15ull * (step * (uint64_t)batch + (uint64_t)i + 1));
        const uint64_t row = i < n_tail_rows ? tail[h % n_tail] : kept[h % n_kept];
        for (int f = 0; f < cols; f++) Xb[(int64_t)i * cols + f] = X[row * cols + f];
        tb[i] = (t[row] - t_mean) * t_inv_sd;
    }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

__global__ void gather_u64_kernel(const uint64_t *__restrict__ src, const uint64_t *__restrict__ pos,
                                  const int32_t *__restrict__ n, uint64_t *__restrict__ dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < *n; i += gridDim.x * blockDim.x) dst[i] = src[pos[i]];
}

// device allocations released on the stream when the scope ends
struct Pool {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Pool(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t get(T **p, size_t count)
    {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count * sizeof(T), 16), st);
        if (e != cudaSuccess) return e;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return cudaSuccess;
    }
    void release(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) { cudaFreeAsync(q, st); q = nullptr; }
    }
    ~Pool()
    {
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, st);
    }
};

epi_status pfail(epi_status s, const char *msg)
{
    set_last_error(msg);
    return s;
}

constexpr int kMaxTriples = 1 << 24;

#define PCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return pfail(e_ == cudaErrorMemoryAllocation ? EPI_ENOMEM : EPI_ECUDA,            \
                         cudaGetErrorString(e_));                                             \
    } while (0)
#define PST(call)                              \
    do {                                       \
        epi_status s_ = (call);                \
        if (s_ != EPI_OK) return s_;           \
    } while (0)

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Exhaustive single-precision scores of orders 1, 2, 3 and, for the
// 30-feature set, 4 (kept with the dataset).
struct Lower {
    const float *s[5] = {};
};

epi_status lower_tables(epi_dataset *ds, Lower &L, bool quad)
{
    for (int k : {1, 2, 3}) PST(epi_dataset_lower_scores(ds, k, &L.s[k]));
    if (quad) {
        const DevData d = epi_dataset_dev(ds);
        size_t free_b = 0, total_b = 0;
        PCK(cudaMemGetInfo(&free_b, &total_b));
        if ((double)host_binom(d.n, 4) * 4.0 > 0.5 * (double)free_b)
            return pfail(EPI_ENOMEM, "proposer: the exhaustive order-4 table of the 30-feature set does not fit in "
                                     "device memory (use the 25-feature set)");
        PST(epi_dataset_lower_scores(ds, 4, &L.s[4]));
    }
    return EPI_OK;
}

// ordered compaction of the marked positions of flags[0, count): per-block
// counts, an exclusive scan, then each block writes its marked positions in
// index order
constexpr int kCompactBlocks = 1024;

__device__ __forceinline__ void compact_range(uint64_t count, uint64_t &b, uint64_t &e)
{
    const uint64_t per = (count + kCompactBlocks - 1) / kCompactBlocks;
    b = (uint64_t)blockIdx.x * per;
    e = b + per < count ? b + per : count;
    if (b > count) b = count;
}

__global__ void __launch_bounds__(256) flag_count_kernel(const uint8_t *__restrict__ flags, uint64_t count,
                                                         unsigned long long *__restrict__ cnt)
{
    __shared__ unsigned long long c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    uint64_t b, e;
    compact_range(count, b, e);
    unsigned long long mine = 0;
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) mine += flags[i];
    atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kCompactBlocks) flag_scan_kernel(unsigned long long *__restrict__ cnt,
                                                                   int32_t *__restrict__ total,
                                                                   unsigned long long *__restrict__ running)
{
    __shared__ unsigned long long s[kCompactBlocks];
    const int t = threadIdx.x;
    const unsigned long long own = cnt[t];
    s[t] = own;
    __syncthreads();
    for (int o = 1; o < kCompactBlocks; o <<= 1) {
        const unsigned long long add = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    cnt[t] = s[t] - own;   // exclusive
    if (t == kCompactBlocks - 1) {
        if (total) *total = (int32_t)s[t];
        if (running) *running += s[t];     // one thread: a running count over calls
    }
}

template <typename T>
__global__ void __launch_bounds__(256) flag_write_kernel(const uint8_t *__restrict__ flags, uint64_t count,
                                                         const unsigned long long *__restrict__ off,
                                                         T *__restrict__ out)
{
    __shared__ uint32_t wsum[8];
    uint64_t b, e;
    compact_range(count, b, e);
    uint64_t base = off[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t i0 = b; i0 < e; i0 += blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        const bool f = i < e && flags[i] != 0;
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        uint64_t before = base;
        for (int w = 0; w < warp; w++) before += wsum[w];
        before += __popc(m & ((1u << lane) - 1u));
        if (f) out[before] = (T)i;
        uint32_t total = 0;
        for (int w = 0; w < 8; w++) total += wsum[w];
        __syncthreads();
        base += total;
    }
}

__global__ void flag_set_kernel(uint8_t *__restrict__ flags, const uint64_t *__restrict__ idx, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        flags[idx[i]] = 1;
}

// The best T triples by (order-3 score desc, rank asc), listed as [T][3] in
// rank order: radix select of the T best, then their ranks marked and
// compacted in index order (deterministic for any T).
epi_status best_triples(epi_dataset *ds, Pool &pool, const float *s3, int T, uint32_t **triples, int *T_out)
{
    epi_ctx *ctx = epi_dataset_ctx(ds);
    cudaStream_t st = epi_ctx_stream(ctx);
    const DevData d = epi_dataset_dev(ds);
    const int64_t total3 = (int64_t)host_binom(d.n, 3);
    T = (int)std::min<int64_t>(T, total3);
    uint64_t *sel, *rk;
    int32_t *nn;
    uint8_t *flags;
    unsigned long long *cnt;
    unsigned char *scratch;
    PCK(pool.get(&sel, T));
    PCK(pool.get(&rk, T));
    PCK(pool.get(&nn, 1));
    PCK(pool.get(&flags, total3));
    PCK(pool.get(&cnt, kCompactBlocks));
    PCK(pool.get(&scratch, topk_scratch_bytes(T)));
    PCK(launch_topk(s3, nullptr, total3, T, scratch, false, nullptr, sel, nn, epi_ctx_num_sms(ctx), st));
    PCK(cudaMemsetAsync(flags, 0, (size_t)total3, st));
    flag_set_kernel<<<grid_for(T), 256, 0, st>>>(flags, sel, T);
    flag_count_kernel<<<kCompactBlocks, 256, 0, st>>>(flags, (uint64_t)total3, cnt);
    flag_scan_kernel<<<1, kCompactBlocks, 0, st>>>(cnt, nullptr, nullptr);
    flag_write_kernel<uint64_t><<<kCompactBlocks, 256, 0, st>>>(flags, (uint64_t)total3, cnt, rk);
    PCK(cudaGetLastError());
    int32_t got = 0;
    PCK(cudaMemcpyAsync(&got, nn, 4, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    T = std::min(T, std::max(got, 0));   // fewer only if scores are NaN
    PCK(pool.get(triples, (size_t)std::max(T, 1) * 3));
    if (T > 0) PCK(launch_unrank(d, 3, rk, T, *triples, st));
    epi_ctx_count_launches(ctx, 12 + 5);
    pool.release(flags);
    *T_out = T;
    return T > 0 ? EPI_OK : pfail(EPI_EINVAL, "proposer: no finite order-3 scores");
}

// Ranking and proposal selection: every ranked score stays in device memory
// (5 bytes per candidate), the budget's R best distinct candidates (ranking
// score desc, candidate index asc) are selected by radix select, every
// proposal is counted and scored exactly in FP32 in slices, and the 4096 best
// by exact FP32 score form the pool that the caller re-scores in FP64.
epi_status rank_and_select(epi_dataset *ds, epi_mlp *net, const DevData &d, const Lower &L, int n_feat,
                           const uint32_t *triples, uint64_t total, uint64_t R, int64_t chunk, Pool &pool,
                           uint64_t **pool_idx, int32_t *n_pool, unsigned long long *kept_out, uint64_t *selected_out,
                           float *pool_floor, int &launches)
{
    epi_ctx *ctx = epi_dataset_ctx(ds);
    cudaStream_t st = epi_ctx_stream(ctx);
    size_t free_b = 0, total_b = 0;
    PCK(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = (size_t)total * 5 + (size_t)chunk * (n_feat * 4 + 4) + (size_t)R * 12 + ((size_t)1 << 30);
    if (need > free_b) return pfail(EPI_ENOMEM, "epi_proposer_search: the candidate space's scores do not fit in device memory");
    float *score, *X;
    uint8_t *keep;
    unsigned long long *kept_dev, *ccnt;
    int32_t *nsel, *nkept;
    uint32_t *kidx;
    uint64_t *sel;
    void *scratch;
    PCK(pool.get(&score, total));
    PCK(pool.get(&keep, total));
    PCK(pool.get(&X, (size_t)chunk * n_feat));
    PCK(pool.get(&kidx, chunk));
    PCK(pool.get(&ccnt, kCompactBlocks));
    PCK(pool.get(&nkept, 1));
    PCK(pool.get(&kept_dev, 1));
    PCK(pool.get(&nsel, 1));
    PCK(pool.get(&sel, R));
    PCK(pool.get(reinterpret_cast<unsigned char **>(&scratch), topk_scratch_bytes(4096)));
    PCK(cudaMemsetAsync(kept_dev, 0, 8, st));
    for (uint64_t first = 0; first < total; first += (uint64_t)chunk) {
        const int64_t cnt = (int64_t)std::min<uint64_t>((uint64_t)chunk, total - first);
        PCK(launch_cand_features5(d, triples, (int64_t)first, cnt, L.s[1], L.s[2], L.s[3], L.s[4], X, keep + first,
                                  nullptr, st));
        if (net) {
            // the network only for the kept rows (a set is ranked once):
            // their chunk positions in order, then gathered and scattered by
            // the fused kernel; where it does not apply, every row
            flag_count_kernel<<<kCompactBlocks, 256, 0, st>>>(keep + first, (uint64_t)cnt, ccnt);
            flag_scan_kernel<<<1, kCompactBlocks, 0, st>>>(ccnt, nkept, kept_dev);
            flag_write_kernel<uint32_t><<<kCompactBlocks, 256, 0, st>>>(keep + first, (uint64_t)cnt, ccnt, kidx);
            PCK(cudaGetLastError());
            launches += 3;
            const epi_status fs = mlp_forward_rows(net, X, cnt, kidx, nkept, score + first);
            if (fs == EPI_EUNSUPPORTED) PST(epi_mlp_forward(net, X, cnt, score + first));
            else PST(fs);
        } else {
            PST(epi_heuristic5(ctx, X, cnt, n_feat, score + first));
            count_kernel<<<grid_for(cnt), 256, 0, st>>>(keep + first, cnt, kept_dev);
            launches += 1;
        }
        launches += 2;
    }
    // the proposals: the R best kept candidates (an unordered set)
    PCK(launch_topk(score, keep, (int64_t)total, (int64_t)R, scratch, false, nullptr, sel, nsel, epi_ctx_num_sms(ctx),
                    st));
    launches += 12;
    int32_t n_sel = 0;
    PCK(cudaMemcpyAsync(kept_out, kept_dev, 8, cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(&n_sel, nsel, 4, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    *selected_out = (uint64_t)n_sel;
    pool.release(score);
    pool.release(X);
    pool.release(keep);
    if (n_sel <= 0) {
        *n_pool = 0;
        return EPI_OK;
    }
    // exact FP32 scores of every proposal (tables counted in registers), in slices
    constexpr int64_t kSlice = (int64_t)1 << 22;
    float *exact;
    uint32_t *pc;
    PCK(pool.get(&exact, n_sel));
    PCK(pool.get(&pc, (size_t)std::min<int64_t>(n_sel, kSlice) * 5));
    for (int64_t off = 0; off < (int64_t)n_sel; off += kSlice) {
        const int64_t c = std::min<int64_t>(kSlice, (int64_t)n_sel - off);
        PCK(launch_candidates5_at(d, triples, sel + off, c, pc, st));
        PCK(launch_score5_f32(d, pc, c, exact + off, epi_ctx_num_sms(ctx), st));
        launches += 2;
    }
    // the pool: the 4096 best proposals by exact FP32 score
    const int kp = std::min(4096, n_sel);
    float *vs;
    uint64_t *pos;
    int32_t *nn;
    PCK(pool.get(&vs, kp));
    PCK(pool.get(&pos, kp));
    PCK(pool.get(&nn, 1));
    PCK(launch_topk(exact, nullptr, (int64_t)n_sel, kp, scratch, true, vs, pos, nn, epi_ctx_num_sms(ctx), st));
    PCK(pool.get(pool_idx, kp));
    gather_u64_kernel<<<(kp + 255) / 256, 256, 0, st>>>(sel, pos, nn, *pool_idx);
    launches += 15;
    PCK(cudaMemcpyAsync(n_pool, nn, 4, cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(pool_floor, vs + kp - 1, 4, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    return EPI_OK;
}

}  // namespace prop
}  // namespace epi

using namespace epi;
using namespace epi::prop;

extern "C" {

epi_status epi_proposer_search(epi_dataset *ds, epi_mlp *net, const epi_proposer_opts *opts, epi_result *out,
                               uint32_t *counts, int32_t *n_out, epi_proposer_stats *stats)
{
    if (!ds || !opts || !out || !n_out) return pfail(EPI_EINVAL, "epi_proposer_search: NULL argument");
    const bool quad = opts->quad_features != 0;
    const int n_feat = quad ? 30 : 25;
    if (net && epi_mlp_num_inputs(net) != n_feat)
        return pfail(EPI_EINVAL, quad ? "epi_proposer_search: the network must take the 30 proposer features"
                                      : "epi_proposer_search: the network must take the 25 proposer features");
    const int R = opts->budget, top_n = opts->top_n;
    if (opts->top_triples < 1 || opts->top_triples > kMaxTriples)
        return pfail(EPI_EINVAL, "epi_proposer_search: top_triples outside 1..2^24");
    if (R < 1 || R > (1 << 30)) return pfail(EPI_EINVAL, "epi_proposer_search: budget outside 1..2^30");
    if (top_n < 1 || top_n > std::min(R, 4096)) return pfail(EPI_EINVAL, "epi_proposer_search: top_n outside 1..min(budget, 4096)");
    const DevData d = epi_dataset_dev(ds);
    if (d.n < 5) return pfail(EPI_EINVAL, "epi_proposer_search: needs at least 5 SNPs");
    epi_ctx *ctx = epi_dataset_ctx(ds);
    cudaStream_t st = epi_ctx_stream(ctx);
    PCK(cudaSetDevice(epi_ctx_device(ctx)));
    *n_out = 0;
    Pool pool(st);
    const double t0 = now_ms();

    // exhaustive lower orders and the expanded triples
    Lower L;
    PST(lower_tables(ds, L, quad));
    uint32_t *triples;
    int T = 0;
    PST(best_triples(ds, pool, L.s[3], opts->top_triples, &triples, &T));
    PCK(cudaStreamSynchronize(st));
    const double t1 = now_ms();

    const uint64_t per = host_binom(d.n - 3, 2);
    const uint64_t total = (uint64_t)T * per;
    const int64_t chunk = (int64_t)std::min<uint64_t>(total, opts->chunk > 0 ? (uint64_t)opts->chunk : (uint64_t)1 << 22);
    int launches = 0;
    // the proposals: candidate indices (device) of the sets re-scored below
    int32_t n_prop = 0;
    unsigned long long kept = 0;
    uint64_t *lr = nullptr;
    uint64_t selected = 0;
    float pool_floor = -INFINITY;     // exact FP32 score of the weakest pooled proposal
    PST(rank_and_select(ds, net, d, L, n_feat, triples, total, (uint64_t)R, chunk, pool, &lr, &n_prop, &kept,
                        &selected, &pool_floor, launches));
    const double t2 = now_ms();

    // exact re-score of the proposals
    std::vector<uint32_t> hc((size_t)std::max(n_prop, 1) * 5);
    std::vector<double> h64(std::max(n_prop, 1));
    std::vector<float> h32(std::max(n_prop, 1));
    std::vector<uint32_t> ht;
    const int cells = 243;
    if (n_prop > 0) {
        uint32_t *pc, *tabs;
        float *f32;
        double *f64;
        PCK(pool.get(&pc, (size_t)n_prop * 5));
        PCK(pool.get(&tabs, (size_t)n_prop * 2 * cells));
        PCK(pool.get(&f32, n_prop));
        PCK(pool.get(&f64, n_prop));
        PCK(launch_candidates5_at(d, triples, lr, n_prop, pc, st));
        PCK(launch_tables(d, 5, pc, n_prop, tabs, epi_ctx_num_sms(ctx), st));
        PCK(launch_score_tables(d, 5, tabs, n_prop, f32, f64, epi_ctx_num_sms(ctx), st));
        launches += 3;
        PCK(cudaMemcpyAsync(hc.data(), pc, (size_t)n_prop * 20, cudaMemcpyDeviceToHost, st));
        PCK(cudaMemcpyAsync(h64.data(), f64, (size_t)n_prop * 8, cudaMemcpyDeviceToHost, st));
        PCK(cudaMemcpyAsync(h32.data(), f32, (size_t)n_prop * 4, cudaMemcpyDeviceToHost, st));
        if (counts) {
            ht.resize((size_t)n_prop * 2 * cells);
            PCK(cudaMemcpyAsync(ht.data(), tabs, ht.size() * 4, cudaMemcpyDeviceToHost, st));
        }
        PCK(cudaStreamSynchronize(st));
    }
    epi_ctx_count_launches(ctx, launches);
    // best top_n by exact score, ties by lexicographic rank
    const uint64_t total5 = host_binom(d.n, 5);
    std::vector<uint64_t> rank5(std::max(n_prop, 1));
    for (int i = 0; i < n_prop; i++) {
        uint64_t s = 0;
        for (int t = 0; t < 5; t++) s += host_binom(d.n - 1 - hc[(size_t)i * 5 + t], 5 - t);
        rank5[i] = total5 - 1 - s;
    }
    std::vector<int> order(n_prop);
    for (int i = 0; i < n_prop; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return h64[a] > h64[b] || (h64[a] == h64[b] && rank5[a] < rank5[b]);
    });
    const int n_res = std::min(top_n, n_prop);
    for (int q = 0; q < n_res; q++) {
        const int i = order[q];
        epi_result r;
        std::memset(&r, 0, sizeof(r));
        for (int t = 0; t < 5; t++) r.snp[t] = hc[(size_t)i * 5 + t];
        r.mi = h64[i];
        r.mi_f32 = h32[i];
        r.order = 5;
        r.rank = rank5[i];
        out[q] = r;
        if (counts) std::memcpy(counts + (size_t)q * 2 * cells, ht.data() + (size_t)i * 2 * cells, (size_t)2 * cells * 4);
    }
    *n_out = n_res;
    const double t3 = now_ms();
    if (stats) {
        stats->candidates = total;
        stats->kept = kept;
        stats->proposals = selected;
        // exact among the proposals: every proposal outside the pool scored at
        // most pool_floor in FP32, so at most pool_floor (1 + eps) exactly
        stats->exact_in_proposals =
            (selected <= (uint64_t)n_prop ||
             (n_res == top_n && h64[order[n_res - 1]] > (double)pool_floor * (1.0 + f32_rel_bound(5, d.m))))
                ? 1
                : 0;
        stats->ms_lower = t1 - t0;
        stats->ms_rank = t2 - t1;
        stats->ms_rescore = t3 - t2;
    }
    return EPI_OK;
}

epi_status epi_proposer_train(epi_mlp *net, epi_dataset *const *datasets, int n_ds, const epi_train_opts *o,
                              float *epoch_loss)
{
    if (!net || !datasets || n_ds < 1 || !o) return pfail(EPI_EINVAL, "epi_proposer_train: bad argument");
    if (o->top_triples < 1 || o->top_triples > kMaxTriples || o->epochs < 1 || o->batch < 1 || o->batch > (1 << 20) ||
        !(o->tail_fraction >= 0.0f && o->tail_fraction <= 1.0f) || !(o->lr > 0.0f) || o->target < 0 ||
        o->target > 1)
        return pfail(EPI_EINVAL, "epi_proposer_train: options out of range");
    const int64_t n_in = epi_mlp_num_inputs(net);
    if (n_in != 25 && n_in != 30)
        return pfail(EPI_EINVAL, "epi_proposer_train: the network must take the 25 or 30 proposer features");
    const bool quad = n_in == 30;
    epi_ctx *ctx = epi_dataset_ctx(datasets[0]);
    cudaStream_t st = epi_ctx_stream(ctx);
    PCK(cudaSetDevice(epi_ctx_device(ctx)));
    for (int i = 0; i < n_ds; i++) {
        if (!datasets[i] || epi_dataset_ctx(datasets[i]) != ctx)
            return pfail(EPI_EINVAL, "epi_proposer_train: datasets must share one context");
        const DevData d = epi_dataset_dev(datasets[i]);
        if (d.n < 5) return pfail(EPI_EINVAL, "epi_proposer_train: every dataset needs at least 5 SNPs");
    }
    Pool pool(st);
    // rows of every dataset: features, labels, keep mask
    std::vector<int64_t> base(n_ds + 1, 0);
    std::vector<int> Ts(n_ds);
    for (int i = 0; i < n_ds; i++) {
        const DevData d = epi_dataset_dev(datasets[i]);
        const int T = (int)std::min<uint64_t>((uint64_t)o->top_triples, host_binom(d.n, 3));
        Ts[i] = T;
        base[i + 1] = base[i] + (int64_t)T * (int64_t)host_binom(d.n - 3, 2);
    }
    const int64_t rows = base[n_ds];
    {
        size_t free_b = 0, total_b = 0;
        PCK(cudaMemGetInfo(&free_b, &total_b));
        if ((size_t)rows * ((size_t)n_in * 4 + 13) + ((size_t)4 << 30) > free_b)
            return pfail(EPI_ENOMEM, "epi_proposer_train: the training rows do not fit in device memory");
    }
    float *X, *t;
    uint8_t *keep;
    PCK(pool.get(&X, (size_t)rows * n_in));
    PCK(pool.get(&t, rows));
    PCK(pool.get(&keep, rows));
    constexpr int kTail = 4096;
    uint64_t *tail;
    PCK(pool.get(&tail, (size_t)n_ds * kTail));
    std::vector<uint64_t> tail_h;
    int launches = 0;
    for (int i = 0; i < n_ds; i++) {
        epi_dataset *ds = datasets[i];
        const DevData d = epi_dataset_dev(ds);
        Pool lp(st);
        Lower L;
        PST(lower_tables(ds, L, quad));
        uint32_t *triples;
        int T = 0;
        PST(best_triples(ds, lp, L.s[3], Ts[i], &triples, &T));
        const int64_t cnt = base[i + 1] - base[i];
        // labels: every row's 5-way table counted and scored exactly (FP32)
        constexpr int64_t kSlice = (int64_t)1 << 22;
        uint32_t *combs;
        PCK(lp.get(&combs, (size_t)std::min<int64_t>(cnt, kSlice) * 5));
        for (int64_t f = 0; f < cnt; f += kSlice) {
            const int64_t c = std::min<int64_t>(cnt - f, kSlice);
            const int64_t at = base[i] + f;
            PCK(launch_cand_features5(d, triples, f, c, L.s[1], L.s[2], L.s[3], L.s[4], X + at * n_in, keep + at, combs,
                                      st));
            PCK(launch_score5_f32(d, combs, c, t + at, epi_ctx_num_sms(ctx), st));
            log_label_kernel<<<grid_for(c), 256, 0, st>>>(t + at, c);
            launches += 3;
        }
        // this dataset's best-labelled kept rows
        const int kt = (int)std::min<int64_t>(kTail, cnt);
        int32_t *nn;
        unsigned char *scratch;
        PCK(lp.get(&nn, 1));
        PCK(lp.get(&scratch, topk_scratch_bytes(kt)));
        PCK(launch_topk(t + base[i], keep + base[i], cnt, kt, scratch, false, nullptr, tail + (size_t)i * kTail, nn,
                        epi_ctx_num_sms(ctx), st));
        launches += 12;
        int32_t got = 0;
        std::vector<uint64_t> ti(kt);
        PCK(cudaMemcpyAsync(&got, nn, 4, cudaMemcpyDeviceToHost, st));
        PCK(cudaMemcpyAsync(ti.data(), tail + (size_t)i * kTail, (size_t)kt * 8, cudaMemcpyDeviceToHost, st));
        PCK(cudaStreamSynchronize(st));
        for (int q = 0; q < got; q++) tail_h.push_back(ti[q] + (uint64_t)base[i]);
    }
    // kept rows (host list of positions), tail list packed
    std::vector<uint8_t> keep_h(rows);
    PCK(cudaMemcpyAsync(keep_h.data(), keep, rows, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    std::vector<uint64_t> kept_h;
    kept_h.reserve((size_t)rows / 2);
    for (int64_t r = 0; r < rows; r++)
        if (keep_h[r]) kept_h.push_back((uint64_t)r);
    if (kept_h.empty()) return pfail(EPI_EINVAL, "epi_proposer_train: no training rows");
    uint64_t *kept;
    PCK(pool.get(&kept, kept_h.size()));
    PCK(cudaMemcpyAsync(kept, kept_h.data(), kept_h.size() * 8, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(tail, tail_h.data(), tail_h.size() * 8, cudaMemcpyHostToDevice, st));
    // standardisation of inputs (kept by the network) and labels
    double *mom;
    PCK(pool.get(&mom, (size_t)2 * (n_in + 1)));
    moments_kernel<<<(unsigned)n_in, 256, 0, st>>>(X, rows, (int)n_in, mom);
    moments_kernel<<<1, 256, 0, st>>>(t, rows, 1, mom + 2 * n_in);
    launches += 2;
    std::vector<double> mh((size_t)2 * (n_in + 1));
    PCK(cudaMemcpyAsync(mh.data(), mom, mh.size() * 8, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    std::vector<float> shift(n_in), scale(n_in);
    for (int f = 0; f < n_in; f++) {
        shift[f] = (float)mh[2 * f];
        scale[f] = (float)(1.0 / std::max(mh[2 * f + 1], 1e-6));
    }
    PST(epi_mlp_set_input_norm(net, shift.data(), scale.data()));
    float t_mean = (float)mh[2 * n_in], t_inv_sd = (float)(1.0 / std::max(mh[2 * n_in + 1], 1e-6));
    if (o->target == 1) {
        // membership of each dataset's best-labelled rows as the label
        PCK(cudaMemsetAsync(t, 0, (size_t)rows * 4, st));
        mark_kernel<<<grid_for((int64_t)tail_h.size()), 256, 0, st>>>(t, tail, (int64_t)tail_h.size());
        launches += 1;
        t_mean = 0.0f;
        t_inv_sd = 1.0f;
    }

    // mini-batch AdamW, cosine learning-rate decay to lr / 20
    const int B = o->batch;
    const int n_tail_rows = (int)std::lround((double)B * o->tail_fraction);
    float *Xb, *tb;
    PCK(pool.get(&Xb, (size_t)B * n_in));
    PCK(pool.get(&tb, B));
    const int64_t steps_per_epoch = std::max<int64_t>(1, (int64_t)kept_h.size() / B);
    const int64_t total_steps = steps_per_epoch * o->epochs;
    int64_t step = 0;
    for (int ep = 0; ep < o->epochs; ep++) {
        double acc = 0.0;
        int nacc = 0;
        for (int64_t s = 0; s < steps_per_epoch; s++, step++) {
            const double frac = (double)step / (double)std::max<int64_t>(1, total_steps - 1);
            const float lr = (float)(o->lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(M_PI * frac))));
            gather_batch_kernel<<<grid_for(B), 256, 0, st>>>(X, t, (int)n_in, kept, kept_h.size(), tail, tail_h.size(),
                                                            B, tail_h.empty() ? 0 : n_tail_rows, o->seed, (uint64_t)step,
                                                            t_mean, t_inv_sd, Xb, tb);
            PCK(cudaGetLastError());
            launches += 1;
            const bool probe = (s % 64 == 63) || s == steps_per_epoch - 1;
            float loss = 0.0f;
            PST(epi_mlp_train_step(net, Xb, tb, B, lr, o->wd, probe ? &loss : nullptr));
            if (probe) { acc += loss; nacc++; }
        }
        if (epoch_loss) epoch_loss[ep] = (float)(acc / std::max(nacc, 1));
    }
    epi_ctx_count_launches(ctx, launches);
    return EPI_OK;
}

}  // extern "C"
