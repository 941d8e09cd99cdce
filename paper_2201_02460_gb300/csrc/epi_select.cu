// Top-N retention (Section 2.4: only the combinations with the highest MI
// are kept) made exact on the GPU:
//   1. merge_lists: the per-CTA candidate lists of the search kernel are
//      merged into one pool ordered by (single-precision score desc, rank asc);
//   2. rescore: every pooled combination is recounted exactly (AND + POPC of
//      its k genotype rows, Section 2.2) and scored in double precision;
//   3. finalize: the pool is sorted by (double MI desc, lexicographic rank
//      asc), the best N are written out, and the margin check proves that no
//      combination outside the pool could have entered the top N (otherwise
//      the host retries with a larger pool).
// Also the table kernels behind epi_tables / epi_score_tables.
#include "epi_internal.cuh"
#include "epi_host.h"

namespace epi {

struct MergeState {
    int32_t list_len, nbuf;
    float thr;
};

__global__ void __launch_bounds__(1024) merge_lists_kernel(const float *__restrict__ ls, const uint64_t *__restrict__ lr,
                                                           const int32_t *__restrict__ lc, int nlists, int stride,
                                                           int pool, int cand_p2, float *__restrict__ out_s,
                                                           uint64_t *__restrict__ out_r, int32_t *__restrict__ out_n,
                                                           float floor)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *rk = reinterpret_cast<uint64_t *>(smem);
    float *sc = reinterpret_cast<float *>(rk + cand_p2);
    __shared__ MergeState S;
    if (threadIdx.x == 0) { S.list_len = 0; S.nbuf = 0; S.thr = floor; }
    __syncthreads();
    const int64_t total = (int64_t)nlists * stride;
    for (int64_t base = 0; base < total; base += blockDim.x) {
        const int64_t e = base + threadIdx.x;
        if (e < total) {
            const int l = (int)(e / stride);
            const int i = (int)(e - (int64_t)l * stride);
            if (i < lc[l]) {
                const float s = ls[e];
                if (s >= S.thr) {
                    const int pos = S.list_len + atomicAdd(&S.nbuf, 1);
                    sc[pos] = s;
                    rk[pos] = lr[e];
                }
            }
        }
        __syncthreads();
        const bool last = base + blockDim.x >= total;
        if (S.nbuf > (int)blockDim.x || (last && S.nbuf > 0)) {
            const int live = S.list_len + S.nbuf;
            const int p2 = next_pow2(live < 2 ? 2 : live);
            for (int i = live + threadIdx.x; i < p2; i += blockDim.x) { sc[i] = floor; rk[i] = ~0ull; }
            __syncthreads();
            block_sort_cands(sc, rk, p2);
            if (threadIdx.x == 0) {
                S.list_len = live < pool ? live : pool;
                S.nbuf = 0;
                if (S.list_len == pool) S.thr = sc[pool - 1];
            }
        }
        __syncthreads();
    }
    const int L = S.list_len;
    for (int i = threadIdx.x; i < L; i += blockDim.x) { out_s[i] = sc[i]; out_r[i] = rk[i]; }
    if (threadIdx.x == 0) *out_n = L;
}

// Exact counts of one combination, cell x = sum_t g_t 3^(k-1-t); one thread
// per (class, cell) pair.
__device__ inline void count_cells(const DevData &d, int k, const int32_t *comb, uint32_t *out)
{
    int cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    for (int idx = threadIdx.x; idx < 2 * cells; idx += blockDim.x) {
        const int half = idx / cells;
        const int x = idx - half * cells;
        const uint32_t *rows[EPI_MAX_ORDER];
        int rem = x, div = cells / 3;
        for (int t = 0; t < k; t++) {
            const int g = rem / div;
            rem -= g * div;
            div = div > 1 ? div / 3 : 1;
            rows[t] = d.masks + ((int64_t)comb[t] * 3 + g) * d.Wt;
        }
        const int wb = half ? d.W1 : 0, we = half ? d.Wt : d.W1;
        uint32_t c = 0;
        for (int w = wb; w < we; w++) {
            uint32_t v = rows[0][w];
            for (int t = 1; t < k; t++) v &= rows[t][w];
            c += __popc(v);
        }
        out[half * cells + x] = c;
    }
}

// double-precision MI of a counted table, cells in ascending order
__device__ inline double table_mi_f64(const DevData &d, const uint32_t *ct, int cells)
{
    double acc = 0.0;
    for (int x = 0; x < cells; x++) {
        const uint32_t a = ct[x], b = ct[cells + x];
        acc += mi_term_f64(a, a + b, d.m1, d.m);
        acc += mi_term_f64(b, a + b, d.m0, d.m);
    }
    return acc / (double)d.m;
}

__device__ inline float table_mi_f32(const DevData &d, const uint32_t *ct, int cells)
{
    const MiConstF32 mc = make_mi_const(d.m, d.m1, d.m0);
    SumF32 acc;
    for (int x = 0; x < cells; x++) acc.add(cell_terms_f32(ct[x], ct[cells + x], mc));
    return __fdiv_rn(acc.value(), mc.fm);
}

constexpr int kRescoreThreads = 256;

// One pooled combination per block: its table, then its double-precision MI
// with the cells shared out over the block (thread t takes cells t, t + 256,
// ...) and the threads' sums added as a tree in a fixed order, so the value
// is the same on every run (the 13,122 terms of an order-8 table took one
// thread 4.8 ms of double-precision divisions and logarithms).
__global__ void __launch_bounds__(kRescoreThreads) rescore_kernel(DevData d, int k,
                                                                  const uint64_t *__restrict__ cand_rank,
                                                                  const int32_t *__restrict__ cand_n,
                                                                  uint32_t *__restrict__ counts,
                                                                  double *__restrict__ mi64, int32_t *__restrict__ combs)
{
    __shared__ int32_t comb[EPI_MAX_ORDER];
    __shared__ double part[kRescoreThreads];
    const int c = blockIdx.x;
    if (c >= *cand_n) return;
    int cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    if (threadIdx.x == 0) {
        unrank_lex(d.binom, d.n, k, cand_rank[c], comb);
        for (int t = 0; t < k; t++) combs[(int64_t)c * k + t] = comb[t];
    }
    __syncthreads();
    uint32_t *ct = counts + (int64_t)c * 2 * cells;
    count_cells(d, k, comb, ct);
    __syncthreads();
    double acc = 0.0;
    for (int x = threadIdx.x; x < cells; x += kRescoreThreads) {
        const uint32_t a = ct[x], b = ct[cells + x];
        acc += mi_term_f64(a, a + b, d.m1, d.m);
        acc += mi_term_f64(b, a + b, d.m0, d.m);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRescoreThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mi64[c] = part[0] / (double)d.m;
}

__device__ __forceinline__ bool final_better(double ma, uint64_t ra, double mb, uint64_t rb)
{
    return ma > mb || (ma == mb && ra < rb);
}

__global__ void __launch_bounds__(1024) finalize_kernel(DevData d, int k, int top_n, int pool,
                                                        const float *__restrict__ cand_s, const uint64_t *__restrict__ cand_r,
                                                        const int32_t *__restrict__ cand_n,
                                                        const double *__restrict__ mi64, const int32_t *__restrict__ combs,
                                                        const uint32_t *__restrict__ counts, const uint32_t *__restrict__ global_thr,
                                                        uint64_t total, epi_result *__restrict__ out,
                                                        uint32_t *__restrict__ out_counts, int32_t *__restrict__ n_out,
                                                        int32_t *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = *cand_n;
    const int p2 = next_pow2(L < 2 ? 2 : L);
    double *key = reinterpret_cast<double *>(smem);
    uint64_t *rk = reinterpret_cast<uint64_t *>(key + p2);
    int32_t *idx = reinterpret_cast<int32_t *>(rk + p2);
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        if (i < L) { key[i] = mi64[i]; rk[i] = cand_r[i]; idx[i] = i; }
        else { key[i] = -1.0; rk[i] = ~0ull; idx[i] = -1; }
    }
    __syncthreads();
    for (int kk = 2; kk <= p2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const bool sw = up ? final_better(key[ixj], rk[ixj], key[i], rk[i])
                                       : final_better(key[i], rk[i], key[ixj], rk[ixj]);
                    if (sw) {
                        double tk = key[i]; key[i] = key[ixj]; key[ixj] = tk;
                        uint64_t tr = rk[i]; rk[i] = rk[ixj]; rk[ixj] = tr;
                        int32_t ti = idx[i]; idx[i] = idx[ixj]; idx[ixj] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int N = L < top_n ? L : top_n;
    int cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int c = idx[i];
        epi_result r;
        for (int t = 0; t < EPI_MAX_ORDER; t++) r.snp[t] = t < k ? (uint32_t)combs[(int64_t)c * k + t] : 0u;
        r.mi = mi64[c];
        r.mi_f32 = cand_s[c];
        r.order = (uint32_t)k;
        r.rank = cand_r[c];
        out[i] = r;
    }
    if (out_counts) {
        for (int64_t e = threadIdx.x; e < (int64_t)N * 2 * cells; e += blockDim.x) {
            const int i = (int)(e / (2 * cells));
            const int q = (int)(e - (int64_t)i * 2 * cells);
            out_counts[e] = counts[(int64_t)idx[i] * 2 * cells + q];
        }
    }
    if (threadIdx.x == 0) {
        *n_out = N;
        // margin check: every combination outside the pool scored at most
        // tau in single precision, hence at most tau / (1 - eps) exactly
        float tau = __uint_as_float(*global_thr);
        if (L == pool && (uint64_t)L < total) tau = fmaxf(tau, cand_s[L - 1]);
        if (tau > 0.0f && N > 0 && (uint64_t)L < total) {
            const double eps = f32_rel_bound(k, d.m);
            const double sigma = key[N - 1];
            if (!((double)tau / (1.0 - eps) < sigma * (1.0 - 1e-12))) atomicOr(status, ST_POOL_OVERFLOW);
        }
    }
}

__global__ void tables_kernel(DevData d, int k, const uint32_t *__restrict__ combs, int64_t count,
                              uint32_t *__restrict__ out)
{
    __shared__ int32_t comb[EPI_MAX_ORDER];
    int cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    for (int64_t c = blockIdx.x; c < count; c += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < k) comb[threadIdx.x] = (int32_t)combs[c * k + threadIdx.x];
        __syncthreads();
        count_cells(d, k, comb, out + c * 2 * cells);
    }
}

__global__ void score_tables_kernel(DevData d, int k, const uint32_t *__restrict__ tabs, int64_t count,
                                    float *__restrict__ f32, double *__restrict__ f64)
{
    int cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < count; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *ct = tabs + c * 2 * cells;
        if (f32) f32[c] = table_mi_f32(d, ct, cells);
        if (f64) f64[c] = table_mi_f64(d, ct, cells);
    }
}

__global__ void publish_status_kernel(const int32_t *__restrict__ bits, int32_t *__restrict__ code)
{
    const int32_t b = *bits;
    int32_t c = EPI_OK;
    if (b & ST_TIMEOUT) c = EPI_ETIMEOUT;
    else if (b & ST_POOL_OVERFLOW) c = EPI_EOVERFLOW;
    else if (b & (ST_BAD_GENO | ST_BAD_PHENO)) c = EPI_EINVAL;
    else if (b) c = EPI_ECUDA;
    *code = c;
}

cudaError_t launch_publish_status(const int32_t *bits, int32_t *code, cudaStream_t st)
{
    publish_status_kernel<<<1, 1, 0, st>>>(bits, code);
    return cudaGetLastError();
}

__global__ void unrank_kernel(DevData d, int k, const uint64_t *__restrict__ ranks, int64_t count,
                              uint32_t *__restrict__ combs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[EPI_MAX_ORDER];
        unrank_lex(d.binom, d.n, k, ranks[i], c);
        for (int t = 0; t < k; t++) combs[i * k + t] = (uint32_t)c[t];
    }
}

cudaError_t launch_unrank(const DevData &d, int k, const uint64_t *ranks, int64_t count, uint32_t *combs,
                          cudaStream_t st)
{
    int64_t g = (count + 255) / 256;
    if (g > 4096) g = 4096;
    unrank_kernel<<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(d, k, ranks, count, combs);
    return cudaGetLastError();
}

size_t merge_smem_bytes(int cand_p2) { return (size_t)cand_p2 * 12; }
size_t finalize_smem_bytes(int pool) { return (size_t)next_pow2(pool < 2 ? 2 : pool) * 20; }

cudaError_t launch_merge(const float *ls, const uint64_t *lr, const int32_t *lc, int nlists, int stride, int pool,
                         float *out_s, uint64_t *out_r, int32_t *out_n, cudaStream_t st, float floor)
{
    const int cand_p2 = next_pow2(pool + 2 * 1024);
    const size_t smem = merge_smem_bytes(cand_p2);
    cudaError_t e = cudaFuncSetAttribute(merge_lists_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    merge_lists_kernel<<<1, 1024, smem, st>>>(ls, lr, lc, nlists, stride, pool, cand_p2, out_s, out_r, out_n, floor);
    return cudaGetLastError();
}

cudaError_t launch_rescore(const DevData &d, int k, int pool, const uint64_t *cand_r, const int32_t *cand_n,
                           uint32_t *counts, double *mi64, int32_t *combs, cudaStream_t st)
{
    rescore_kernel<<<pool, kRescoreThreads, 0, st>>>(d, k, cand_r, cand_n, counts, mi64, combs);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevData &d, int k, int top_n, int pool, const float *cand_s, const uint64_t *cand_r,
                            const int32_t *cand_n, const double *mi64, const int32_t *combs, const uint32_t *counts,
                            const uint32_t *global_thr, uint64_t total, epi_result *out, uint32_t *out_counts,
                            int32_t *n_out, int32_t *status, cudaStream_t st)
{
    const size_t smem = finalize_smem_bytes(pool);
    cudaError_t e = cudaFuncSetAttribute(finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, 1024, smem, st>>>(d, k, top_n, pool, cand_s, cand_r, cand_n, mi64, combs, counts, global_thr,
                                           total, out, out_counts, n_out, status);
    return cudaGetLastError();
}

cudaError_t launch_tables(const DevData &d, int k, const uint32_t *combs, int64_t count, uint32_t *out, int num_sms,
                          cudaStream_t st)
{
    int64_t g = count < (int64_t)num_sms * 8 ? count : (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    tables_kernel<<<(unsigned)g, 256, 0, st>>>(d, k, combs, count, out);
    return cudaGetLastError();
}

cudaError_t launch_score_tables(const DevData &d, int k, const uint32_t *tabs, int64_t count, float *f32, double *f64,
                                int num_sms, cudaStream_t st)
{
    int64_t g = (count + 255) / 256;
    if (g > num_sms * 4) g = num_sms * 4;
    if (g < 1) g = 1;
    score_tables_kernel<<<(unsigned)g, 256, 0, st>>>(d, k, tabs, count, f32, f64);
    return cudaGetLastError();
}

// Exact single-precision MI of order-5 sets without materialising their
// tables (Section 2.2 counts, Eq. 1-3 in the cancellation-free form): one
// warp per set.  The set's 15 genotype rows are staged in shared memory in
// chunks of kS5Ch words (rows padded to an odd stride, so lanes reading the
// three genotype rows of one SNP hit distinct banks); lane l owns the
// four-SNP prefixes p = l, l + 32, l + 64 (p < 81; the lanes past 81 repeat
// prefix 0 and discard it) and, per word, counts popc(prefix & last-SNP
// genotype g) into case or control counters (the class of a word is uniform
// across the warp).  Cell x = 3 p + g; each lane sums the terms of its cells,
// the warp sums the lanes.  The summation order differs from the serial
// table sum, inside the same FP32 error bound.
constexpr int kS5Warps = 8, kS5Ch = 64, kS5Pad = kS5Ch + 1;

__global__ void __launch_bounds__(kS5Warps * 32) score5_f32_kernel(DevData d, const uint32_t *__restrict__ combs,
                                                                  int64_t count, float *__restrict__ out)
{
    __shared__ uint32_t rows[kS5Warps][15][kS5Pad];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t(*R)[kS5Pad] = rows[warp];
    const MiConstF32 mc = make_mi_const(d.m, d.m1, d.m0);
    const int Wt = d.Wt, W1 = d.W1;
    // the lane's prefixes: row index t * 3 + g_t of the four prefix SNPs
    int off[3][4];
    bool valid[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int p0 = lane + 32 * j;
        valid[j] = p0 < 81;
        const int p = valid[j] ? p0 : 0;
        off[j][0] = p / 27;
        off[j][1] = 3 + (p / 9) % 3;
        off[j][2] = 6 + (p / 3) % 3;
        off[j][3] = 9 + p % 3;
    }
    for (int64_t s = (int64_t)blockIdx.x * kS5Warps + warp; s < count; s += (int64_t)gridDim.x * kS5Warps) {
        const uint32_t *src[5];
#pragma unroll
        for (int t = 0; t < 5; t++) src[t] = d.masks + (int64_t)combs[s * 5 + t] * 3 * Wt;
        uint32_t cc[3][3] = {}, ck[3][3] = {};
        for (int c0 = 0; c0 < Wt; c0 += kS5Ch) {
            const int cw = min(kS5Ch, Wt - c0);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 15; r++)
                for (int w = lane; w < cw; w += 32) R[r][w] = src[r / 3][(r % 3) * Wt + c0 + w];
            __syncwarp();
            const int split = min(max(W1 - c0, 0), cw);   // words [0, split) are cases
            auto word = [&](int w, uint32_t (&acc)[3][3]) {
                const uint32_t l0 = R[12][w], l1 = R[13][w], l2 = R[14][w];
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const uint32_t pw = R[off[j][0]][w] & R[off[j][1]][w] & R[off[j][2]][w] & R[off[j][3]][w];
                    acc[j][0] += __popc(pw & l0);
                    acc[j][1] += __popc(pw & l1);
                    acc[j][2] += __popc(pw & l2);
                }
            };
            for (int w = 0; w < split; w++) word(w, cc);
            for (int w = split; w < cw; w++) word(w, ck);
        }
        SumF32 acc;
#pragma unroll
        for (int j = 0; j < 3; j++)
            if (valid[j]) {
#pragma unroll
                for (int g = 0; g < 3; g++) acc.add(cell_terms_f32(cc[j][g], ck[j][g], mc));
            }
        float v = acc.value();
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) out[s] = __fdiv_rn(v, mc.fm);
    }
}

cudaError_t launch_score5_f32(const DevData &d, const uint32_t *combs, int64_t count, float *out, int num_sms,
                              cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t g = (count + kS5Warps - 1) / kS5Warps;
    if (g > (int64_t)num_sms * 6) g = (int64_t)num_sms * 6;
    score5_f32_kernel<<<(unsigned)g, kS5Warps * 32, 0, st>>>(d, combs, count, out);
    return cudaGetLastError();
}

// Ranks rank_base + i of the scores at or above thr (any order), appended
// while they fit in `cap`; *n counts all of them.
__global__ void select_ge_kernel(const float *__restrict__ scores, int64_t count, float thr, uint64_t rank_base,
                                 uint64_t *__restrict__ out, uint64_t cap, unsigned long long *__restrict__ n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = scores[i];
        if (v >= thr) {
            const unsigned long long at = atomicAdd(n, 1ull);
            if (at < cap) out[at] = rank_base + (uint64_t)i;
        }
    }
}

cudaError_t launch_select_ge(const float *scores, int64_t count, float thr, uint64_t rank_base, uint64_t *out,
                             uint64_t cap, unsigned long long *n, int num_sms, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t g = (count + 255) / 256;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    select_ge_kernel<<<(unsigned)g, 256, 0, st>>>(scores, count, thr, rank_base, out, cap, n);
    return cudaGetLastError();
}

}  // namespace epi
