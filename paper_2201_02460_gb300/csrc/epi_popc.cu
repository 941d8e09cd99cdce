// Popcount counting path of the exhaustive search.
//
// Section 2.4 / Algorithm 1: combinations are visited prefix by prefix; the
// genotype table of the (k-1)-prefix (Section 2.1, Listing A.1 semantics:
// row-wise AND) is built once into shared memory and reused for every last
// SNP j; the last level is never stored but fused with the population count
// (Section 2.2, Listing A.2 semantics).  The score is the single-precision MI
// of Eq. 1-3 (Section 2.3) and only the best candidates are kept
// (Section 2.4).
//
// GPU mapping:
//   * persistent grid; CTA b owns the contiguous lexicographic rank range
//     [R_b, R_{b+1}) (every combination costs the same, so a static split
//     balances); it unranks R_b once and then steps prefixes in lex order;
//   * a sub-tile is up to T consecutive ranks spanning at most `slots`
//     prefixes; their tables are staged in shared memory as uint4 rows;
//   * one thread per combination: 128-bit loads of the last SNP's rows for
//     genotypes 0 and 1, AND + POPC against every prefix row; genotype 2 is
//     the prefix row's total minus the other two (exact, saves a third of
//     the work);
//   * the counts never leave registers: MI is evaluated in the same thread
//     and compared against the CTA's current threshold; survivors go to a
//     shared-memory buffer that is merged into the CTA's sorted list;
//   * orders 6-8: the same kernel with one warp per combination; at orders
//     7-8 the prefix table (729 or 2187 rows) is materialised in a per-CTA
//     global buffer (the paper's stored `combine` table, Section 2.1), read
//     through L1/L2 by the CTA's threads, which walk the same prefix rows
//     (batched launches keep it in shared memory where it fits).
#include "epi_internal.cuh"
#include "epi_host.h"

namespace epi {

__host__ __device__ constexpr int ipow3(int k) { return k <= 0 ? 1 : 3 * ipow3(k - 1); }

// Words between consecutive rows of a staged prefix table (orders 1-5).
// Orders 6-8 read the table with one lane per row (a warp per combination)
// and store it transposed by 16-byte words instead: uint4 u of row r at
// [u][r], so the 32 lanes' loads of one word position are 512 contiguous
// bytes (coalesced from global memory, conflict-free in shared memory).
__host__ __device__ inline int popc_row_stride(int k, int32_t Wt) { (void)k; return Wt; }

// One dataset of a launch.  A launch may cover several datasets of the same
// order (batched search): CTAs [cta_begin, cta_begin + cta_count) of the grid
// search this dataset's rank range, sized in proportion to its work.
struct PopcDs {
    DevData d;
    uint64_t rank_begin, rank_end;  // lexicographic range searched
    int32_t cta_begin, cta_count;
    uint32_t *global_thr;           // float bits of max over its CTAs of their pool-th score
};

struct PopcParams {
    PopcDs one;                     // the dataset when the launch has one
    const PopcDs *many;             // else [n_ds] in device memory
    const int32_t *cta_ds;          // and the dataset of each CTA
    int32_t tile;                   // combinations per sub-tile (T)
    int32_t pool;                   // list entries kept per CTA
    int32_t slots;                  // prefixes staged per sub-tile
    int32_t cand_p2;                // shared candidate arrays (power of two)
    int32_t max_wt;                 // largest Wt of the launch (shared-memory layout)
    float *list_score;              // [grid][pool]
    uint64_t *list_rank;            // [grid][pool]
    int32_t *list_count;            // [grid]
    float *all_scores;              // optional: every score, [rank - rank_begin] (single dataset)
    uint32_t *pre_global;           // global prefix tables: [grid][pre_cta_words] (global-prefix kernels)
    int64_t pre_cta_words;
    uint32_t *pair_sing;            // (k-2)-prefix kernel: single-count tables [grid][pair_sing_words], or NULL
    int64_t pair_sing_words;
    int32_t top_n;                  // (k-2)-prefix kernel: records asked for (0: not known)
};

struct SlotInfo {
    int64_t base;     // rank of the prefix's first combination (j = s_last + 1)
    int32_t s_last;   // last prefix SNP (-1 for order 1)
    int32_t N;        // number of last SNPs: n - 1 - s_last
    int32_t snp[kMaxOrderGpu];
};

struct SubtileState {
    int64_t F, F_end;              // current sub-tile [F, F_end)
    int64_t cur_base;
    int32_t cur_prefix[kMaxOrderGpu];
    int32_t nslots;
    int32_t list_len, nbuf;
    float thr;
    int32_t done;
};

// next (k-1)-subset of [0, n-1) in lex order; false after the last
__device__ inline bool next_prefix(int32_t *p, int km1, int64_t n)
{
    const int64_t u = n - 1;           // the last SNP needs room after the prefix
    int t = km1 - 1;
    while (t >= 0 && p[t] == u - km1 + t) t--;
    if (t < 0) return false;
    p[t]++;
    for (int v = t + 1; v < km1; v++) p[v] = p[v - 1] + 1;
    return true;
}

__device__ __forceinline__ uint32_t popc4(uint4 p, uint4 a)
{
    return __popc(p.x & a.x) + __popc(p.y & a.y) + __popc(p.z & a.z) + __popc(p.w & a.w);
}

// Counts of one combination against R staged prefix rows, over words [wb, we).
template <int R>
__device__ __forceinline__ void count_rows(const uint32_t *__restrict__ pre, int Wt, const uint32_t *__restrict__ mj,
                                           int wb, int we, uint32_t (&c0)[R], uint32_t (&c1)[R])
{
#pragma unroll
    for (int r = 0; r < R; r++) { c0[r] = 0; c1[r] = 0; }
#pragma unroll 2
    for (int w = wb; w < we; w += 4) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(mj + w));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(mj + Wt + w));
#pragma unroll
        for (int r = 0; r < R; r++) {
            const uint4 p = *reinterpret_cast<const uint4 *>(pre + r * Wt + w);
            c0[r] += popc4(p, a);
            c1[r] += popc4(p, b);
        }
    }
}

// Single-precision MI of one combination: the prefix rows are taken R at a
// time (R counters per genotype and class stay in registers); genotype 2 of
// the last SNP is the prefix row's total minus genotypes 0 and 1.
template <int K, int R>
__device__ __forceinline__ float score_popc(const uint32_t *__restrict__ pre, const uint32_t *__restrict__ tot,
                                            const uint32_t *__restrict__ mj, const DevData &d, const MiConstF32 &mc)
{
    constexpr int PR = ipow3(K - 1);
    constexpr int G = PR / R;
    static_assert(PR % R == 0, "row group must divide the prefix rows");
    SumF32 acc;
#pragma unroll 1
    for (int grp = 0; grp < G; grp++) {
        const uint32_t *pg = pre + grp * R * d.Wt;
        uint32_t a0[R], a1[R], b0[R], b1[R];
        count_rows<R>(pg, d.Wt, mj, 0, d.W1, a0, a1);
        count_rows<R>(pg, d.Wt, mj, d.W1, d.Wt, b0, b1);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const uint32_t t1 = tot[(grp * R + r) * 2 + 0];
            const uint32_t t0 = tot[(grp * R + r) * 2 + 1];
            acc.add(cell_terms_f32(a0[r], b0[r], mc));
            acc.add(cell_terms_f32(a1[r], b1[r], mc));
            acc.add(cell_terms_f32(t1 - a0[r] - a1[r], t0 - b0[r] - b1[r], mc));
        }
    }
    return __fdiv_rn(acc.value(), mc.fm);
}

// Sort the live list + buffer, keep the best `pool`, refresh the threshold.
__device__ inline void flush_list(SubtileState &S, float *sc, uint64_t *rk, int pool, int cand_p2,
                                  uint32_t *global_thr)
{
    __syncthreads();
    const int live = S.list_len + S.nbuf;
    const int p2 = next_pow2(live < 2 ? 2 : live);
    for (int i = live + threadIdx.x; i < p2 && i < cand_p2; i += blockDim.x) { sc[i] = -1.0f; rk[i] = ~0ull; }
    __syncthreads();
    block_sort_cands(sc, rk, p2);
    if (threadIdx.x == 0) {
        S.list_len = live < pool ? live : pool;
        S.nbuf = 0;
        if (S.list_len == pool) {
            const float t = sc[pool - 1];
            S.thr = t;
            atomicMax(global_thr, __float_as_uint(t));
        }
    }
    __syncthreads();
}

// A CTA holding at least top_n candidates knows that top_n combinations
// score at least its top_n-th best s, so none below s can enter the top N:
// after a flush it lowers s by its single-precision error bound (four times
// over, so that the final margin check still clears it), and raises its own
// and the global threshold to it.
__device__ inline void publish_top_n(SubtileState &S, float *sc, uint64_t *rk, int pool, int cand_p2,
                                     uint32_t *global_thr, int top_n, int k, int64_t m)
{
    flush_list(S, sc, rk, pool, cand_p2, global_thr);
    if (threadIdx.x == 0 && top_n <= S.list_len) {
        const float t = sc[top_n - 1] * (float)(1.0 - 4.0 * f32_rel_bound(k, m));
        if (t > 0.0f) {
            S.thr = fmaxf(S.thr, t);
            atomicMax(global_thr, __float_as_uint(t));
        }
    }
    __syncthreads();
}

// Exact FP32 MI of one combination by one warp (orders 6-8): lane l takes
// the prefix rows l, l + 32, ... four at a time, counts them against the last
// SNP's genotype-0/1 rows (the same words for every lane: broadcast loads),
// derives genotype 2 from the row totals, sums its cell terms, and the warp
// adds the lanes' sums.
template <int K>
__device__ __forceinline__ float score_popc_warp(const uint32_t *__restrict__ pre,
                                                 const uint32_t *__restrict__ tot, const uint32_t *__restrict__ mj,
                                                 const DevData &d, const MiConstF32 &mc, int lane)
{
    constexpr int PR = ipow3(K - 1);
    SumF32 acc;
    // the table is transposed by uint4: word group u of row r at uint4 u PR + r
    const uint4 *T = reinterpret_cast<const uint4 *>(pre);
#pragma unroll 1
    for (int r0 = lane; r0 < PR; r0 += 4 * 32) {
        const uint4 *rp[4];
#pragma unroll
        for (int i = 0; i < 4; i++) rp[i] = T + min(r0 + 32 * i, PR - 1);
        uint32_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, b0[4] = {0, 0, 0, 0}, b1[4] = {0, 0, 0, 0};
#pragma unroll 2
        for (int w = 0; w < d.W1; w += 4) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(mj + w));
            const uint4 y = __ldg(reinterpret_cast<const uint4 *>(mj + d.Wt + w));
            const size_t off = (size_t)(w >> 2) * PR;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint4 p = rp[i][off];
                a0[i] += popc4(p, x);
                a1[i] += popc4(p, y);
            }
        }
#pragma unroll 2
        for (int w = d.W1; w < d.Wt; w += 4) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(mj + w));
            const uint4 y = __ldg(reinterpret_cast<const uint4 *>(mj + d.Wt + w));
            const size_t off = (size_t)(w >> 2) * PR;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint4 p = rp[i][off];
                b0[i] += popc4(p, x);
                b1[i] += popc4(p, y);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int r = r0 + 32 * i;
            if (r < PR) {
                const uint32_t t1 = tot[r * 2 + 0], t0 = tot[r * 2 + 1];
                acc.add(cell_terms_f32(a0[i], b0[i], mc));
                acc.add(cell_terms_f32(a1[i], b1[i], mc));
                acc.add(cell_terms_f32(t1 - a0[i] - a1[i], t0 - b0[i] - b1[i], mc));
            }
        }
    }
    float v = acc.value();
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return __fdiv_rn(v, mc.fm);
}

template <int K, int R, bool GP>
__global__ void __launch_bounds__(128) popc_search_kernel(PopcParams P)
{
    constexpr int PR = ipow3(K - 1);
    constexpr bool kWarpPerComb = K >= 6;
    const PopcDs &D = P.many ? P.many[P.cta_ds[blockIdx.x]] : P.one;
    const DevData d = D.d;
    const int rstride = popc_row_stride(K, d.Wt);
    const int slot_words = PR * rstride + 4;   // 16-byte skew: slots start on different banks
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: prefix rows (unless global) | totals | candidate scores | candidate ranks
    const size_t pre_words = GP ? 0 : (size_t)P.slots * (PR * popc_row_stride(K, P.max_wt) + 4);
    uint32_t *pre = GP ? P.pre_global + (size_t)blockIdx.x * (size_t)P.pre_cta_words
                       : reinterpret_cast<uint32_t *>(smem);
    uint32_t *tot = reinterpret_cast<uint32_t *>(smem) + pre_words;
    uint64_t *rk = reinterpret_cast<uint64_t *>(smem + (((pre_words + (size_t)P.slots * PR * 2) * 4 + 15) & ~(size_t)15));
    float *sc = reinterpret_cast<float *>(rk + P.cand_p2);
    __shared__ SlotInfo slot[8];
    __shared__ SubtileState S;

    const int km1 = K - 1;
    const MiConstF32 mc = make_mi_const(d.m, d.m1, d.m0);
    const uint64_t span = D.rank_end - D.rank_begin;
    const uint64_t cb = blockIdx.x - (uint64_t)D.cta_begin, cn = (uint64_t)D.cta_count;
    const int64_t R_b = (int64_t)(D.rank_begin + (uint64_t)(((unsigned __int128)span * cb) / cn));
    const int64_t R_e = (int64_t)(D.rank_begin + (uint64_t)(((unsigned __int128)span * (cb + 1)) / cn));

    if (threadIdx.x == 0) {
        S.list_len = 0; S.nbuf = 0; S.thr = -1.0f; S.done = R_b >= R_e;
        S.F = R_b;
        if (!S.done) {
            int32_t c[kMaxOrderGpu];
            unrank_lex(d.binom, d.n, K, (uint64_t)R_b, c);
            const int32_t s_last = K > 1 ? c[K - 2] : -1;
            for (int t = 0; t < km1; t++) S.cur_prefix[t] = c[t];
            S.cur_base = R_b - (c[K - 1] - (s_last + 1));
        }
    }
    __syncthreads();

    while (!S.done) {
        // ---- assemble the sub-tile's prefixes ----------------------------
        if (threadIdx.x == 0) {
            const int64_t lim = min((int64_t)S.F + P.tile, R_e);
            int32_t p[kMaxOrderGpu];
            for (int t = 0; t < km1; t++) p[t] = S.cur_prefix[t];
            int64_t base = S.cur_base;
            int ns = 0;
            bool more = true;
            while (true) {
                SlotInfo &sl = slot[ns];
                sl.base = base;
                sl.s_last = km1 > 0 ? p[km1 - 1] : -1;
                sl.N = (int32_t)(d.n - 1 - sl.s_last);
                for (int t = 0; t < km1; t++) sl.snp[t] = p[t];
                ns++;
                base += sl.N;
                if (base >= lim || ns == P.slots) break;
                if (km1 == 0 || !next_prefix(p, km1, d.n)) { more = false; break; }
            }
            const SlotInfo &last = slot[ns - 1];
            const int64_t last_end = last.base + last.N;
            S.F_end = min(lim, last_end);
            S.nslots = ns;
            // prefix containing the next sub-tile's first rank
            if (S.F_end == last_end && S.F_end < R_e) {
                for (int t = 0; t < km1; t++) p[t] = last.snp[t];
                if (km1 > 0) more = next_prefix(p, km1, d.n);
                for (int t = 0; t < km1; t++) S.cur_prefix[t] = p[t];
                S.cur_base = last_end;
                (void)more;
            } else {
                for (int t = 0; t < km1; t++) S.cur_prefix[t] = last.snp[t];
                S.cur_base = last.base;
            }
            // stricter of the CTA threshold and the best known global one
            const float g = __uint_as_float(*(volatile uint32_t *)D.global_thr);
            if (S.list_len == P.pool || g > 0.0f) S.thr = fmaxf(S.thr, g);
        }
        __syncthreads();

        // ---- stage prefix tables: row x' = sum_t g_t 3^(k-2-t) -------------
        const int ns = S.nslots;
        const int W4 = d.Wt >> 2;
        if constexpr (K >= 6) {
            // blocks of 9 rows that share the genotypes of the first k-3
            // prefix SNPs: their AND is formed once, then the last two SNPs'
            // rows (k + 3 loads per 9 rows instead of 9 (k - 1))
            constexpr int PB = PR / 9;
            // block index fastest: consecutive threads write consecutive rows
            // of one word group of the transposed table
            for (int idx = threadIdx.x; idx < ns * PB * W4; idx += blockDim.x) {
                const int blk = idx % PB;
                const int w4 = (idx / PB) % W4;
                const int s = idx / (W4 * PB);
                uint4 base = make_uint4(~0u, ~0u, ~0u, ~0u);
                int rem = blk;
                int div = PB / 3;
#pragma unroll
                for (int t = 0; t < km1 - 2; t++) {
                    const int g = rem / div;
                    rem -= g * div;
                    div = div > 1 ? div / 3 : 1;
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(
                        d.masks + ((int64_t)slot[s].snp[t] * 3 + g) * d.Wt) + w4);
                    base.x &= v.x; base.y &= v.y; base.z &= v.z; base.w &= v.w;
                }
                const uint4 *ma = reinterpret_cast<const uint4 *>(d.masks + (int64_t)slot[s].snp[km1 - 2] * 3 * d.Wt);
                const uint4 *mb = reinterpret_cast<const uint4 *>(d.masks + (int64_t)slot[s].snp[km1 - 1] * 3 * d.Wt);
                uint4 lb[3];
#pragma unroll
                for (int h = 0; h < 3; h++) lb[h] = __ldg(mb + h * W4 + w4);
                uint4 *ps = reinterpret_cast<uint4 *>(pre + (size_t)s * slot_words) + (size_t)w4 * PR + blk * 9;
#pragma unroll
                for (int g = 0; g < 3; g++) {
                    const uint4 a = __ldg(ma + g * W4 + w4);
                    const uint4 b1 = make_uint4(base.x & a.x, base.y & a.y, base.z & a.z, base.w & a.w);
#pragma unroll
                    for (int h = 0; h < 3; h++)
                        ps[g * 3 + h] = make_uint4(b1.x & lb[h].x, b1.y & lb[h].y, b1.z & lb[h].z, b1.w & lb[h].w);
                }
            }
        } else
        for (int idx = threadIdx.x; idx < ns * PR * W4; idx += blockDim.x) {
            const int w4 = idx % W4;
            const int row = (idx / W4) % PR;
            const int s = idx / (W4 * PR);
            uint4 acc;
            if (K == 1) {
                // the empty prefix: every real individual of each subtable
                const int w = w4 * 4;
                uint32_t v[4];
                for (int q = 0; q < 4; q++) {
                    const int ww = w + q;
                    const int64_t first = ww < d.W1 ? (int64_t)ww * 32 : (int64_t)(ww - d.W1) * 32;
                    const int64_t size = ww < d.W1 ? d.m1 : d.m0;
                    const int64_t left = size - first;
                    v[q] = left >= 32 ? 0xffffffffu : (left <= 0 ? 0u : ((1u << left) - 1u));
                }
                acc = make_uint4(v[0], v[1], v[2], v[3]);
            } else {
                acc = make_uint4(~0u, ~0u, ~0u, ~0u);
                int rem = row;
                int div = PR / 3;
#pragma unroll
                for (int t = 0; t < km1; t++) {
                    const int g = rem / div;
                    rem -= g * div;
                    div = div > 1 ? div / 3 : 1;
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(
                        d.masks + ((int64_t)slot[s].snp[t] * 3 + g) * d.Wt) + w4);
                    acc.x &= v.x; acc.y &= v.y; acc.z &= v.z; acc.w &= v.w;
                }
            }
            reinterpret_cast<uint4 *>(pre + (size_t)s * slot_words + (size_t)row * rstride)[w4] = acc;
        }
        __syncthreads();
        // per-row totals of each subtable (the third genotype by subtraction);
        // orders 6-8: one thread per (row, subtable) of the transposed table,
        // consecutive threads on consecutive rows
        if constexpr (K >= 6) {
            for (int idx = threadIdx.x; idx < ns * PR * 2; idx += blockDim.x) {
                const int row = idx % PR;
                const int half = (idx / PR) & 1;
                const int s = idx / (PR * 2);
                const uint4 *T = reinterpret_cast<const uint4 *>(pre + (size_t)s * slot_words) + row;
                const int ub = half ? d.W1 / 4 : 0, ue = half ? d.Wt / 4 : d.W1 / 4;
                uint32_t c = 0;
                for (int u = ub; u < ue; u++) {
                    const uint4 v = T[(size_t)u * PR];
                    c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                }
                tot[((size_t)s * PR + row) * 2 + half] = c;
            }
        } else
        for (int idx = threadIdx.x; idx < ns * PR * 2; idx += blockDim.x) {
            const int half = idx & 1;
            const int sr = idx >> 1;
            const uint32_t *row = pre + (size_t)(sr / PR) * slot_words + (size_t)(sr % PR) * rstride;
            uint32_t c = 0;
            const int wb = half ? d.W1 : 0, we = half ? d.Wt : d.W1;
            for (int w = wb; w < we; w++) c += __popc(row[w]);
            tot[sr * 2 + half] = c;
        }
        __syncthreads();

        // ---- count and score: one thread per combination -------------------
        const int64_t F = S.F, F_end = S.F_end;
        const int list_len = S.list_len;
        const float thr = S.thr;
        if constexpr (kWarpPerComb) {
            // one warp per combination
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int64_t f = F + warp; f < F_end; f += blockDim.x >> 5) {
                int s = 0;
                while (s + 1 < ns && f >= slot[s + 1].base) s++;
                const int32_t j = slot[s].s_last + 1 + (int32_t)(f - slot[s].base);
                const float score = score_popc_warp<K>(pre + (size_t)s * slot_words, tot + s * PR * 2,
                                                       d.masks + (int64_t)j * 3 * d.Wt, d, mc, lane);
                if (lane == 0) {
                    if (P.all_scores) P.all_scores[f - (int64_t)D.rank_begin] = score;
                    if (score >= thr) {
                        const int pos = list_len + atomicAdd(&S.nbuf, 1);
                        sc[pos] = score;
                        rk[pos] = (uint64_t)f;
                    }
                }
            }
        } else
        for (int64_t f = F + threadIdx.x; f < F_end; f += blockDim.x) {
            int s = 0;
            while (s + 1 < ns && f >= slot[s + 1].base) s++;
            const int32_t j = slot[s].s_last + 1 + (int32_t)(f - slot[s].base);
            const float score = score_popc<K, R>(pre + (size_t)s * slot_words, tot + s * PR * 2,
                                                 d.masks + (int64_t)j * 3 * d.Wt, d, mc);
            if (P.all_scores) P.all_scores[f - (int64_t)D.rank_begin] = score;
            if (score >= thr) {
                const int pos = list_len + atomicAdd(&S.nbuf, 1);
                sc[pos] = score;
                rk[pos] = (uint64_t)f;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.F = F_end;
            S.done = F_end >= R_e;
        }
        __syncthreads();
        if (S.nbuf > P.tile || (S.done && S.nbuf > 0)) flush_list(S, sc, rk, P.pool, P.cand_p2, D.global_thr);
    }
    __syncthreads();
    const int L = S.list_len;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        P.list_score[(size_t)blockIdx.x * P.pool + i] = sc[i];
        P.list_rank[(size_t)blockIdx.x * P.pool + i] = rk[i];
    }
    if (threadIdx.x == 0) P.list_count[blockIdx.x] = L;
}

// ---------------------------------------------------------------------------
// Orders 7-8 with the (k-2)-prefix table in shared memory.
//
// Combinations that share their first k-2 SNPs are consecutive in
// lexicographic order, their last two SNPs (j1 < j2) running over the pairs
// after the prefix.  The prefix's table (3^(k-2) = 243 or 729 rows, Section
// 2.1) is built once in shared memory, transposed by 16-byte words, with its
// row totals and a single-count table: per row, class and SNP j after the
// prefix, the counts of row & j's genotype-0 and genotype-1 rows (in a
// per-CTA global buffer, built once per prefix and shared by the L - 1 pairs
// that contain j).  Each warp then counts one pair at a time, lanes over the
// rows: per row and class the four joint counts n[g1][g2] (g1, g2 in {0, 1}:
// the prefix row AND both last SNPs' genotype rows); the other five cells
// follow by subtraction (n[g1][2] = row & j1:g1 minus n[g1][0] + n[g1][1],
// and so on, n[2][2] from the row total).  The prefix table never leaves the
// SM, and it serves C(L, 2) combinations (L = SNPs after the prefix) instead
// of L.
// threads per CTA and prefix rows per lane and block (tuning parameters;
// measured on the order-8 Table-2 workload: 4 rows x 256 threads 104 ms
// (239 registers, 8 warps per SM), 2 x 384 65 ms, 2 x 512 63 ms, 1 x 512
// 57.6 ms, 1 x 768 52.3 ms, 1 x 1024 52.0 ms (64 registers): the counting
// loop is latency-bound, and more warps hide it)
#ifndef EPI_PAIR_THREADS
#define EPI_PAIR_THREADS 1024
#endif
#ifndef EPI_PAIR_ROWS
#define EPI_PAIR_ROWS 1
#endif
// lowest order searched with the (k-2)-prefix kernel (tuning parameter;
// order 6, 60 SNPs x 2048: 690 ms against 961 ms for the (k-1)-prefix
// kernel, whose 243-row tables leave one 4-warp CTA per SM)
#ifndef EPI_PAIR_MIN_ORDER
#define EPI_PAIR_MIN_ORDER 6
#endif
constexpr int kPairThreads = EPI_PAIR_THREADS;
constexpr int kPairRows = EPI_PAIR_ROWS;
constexpr int kPairChunk = 256;   // pairs counted between candidate-buffer checks

__host__ __device__ inline size_t pair_table_bytes(int k, int32_t Wt)
{
    const size_t PR = (size_t)ipow3(k - 2);
    return (size_t)(Wt / 4) * PR * 16 + PR * 2 * 4;
}

__host__ __device__ inline int pair_cand_p2(int pool) { return next_pow2(pool + 2 * kPairChunk); }

__host__ __device__ inline size_t pair_smem_bytes(int k, int32_t Wt, int pool)
{
    return ((pair_table_bytes(k, Wt) + 15) & ~(size_t)15) + (size_t)pair_cand_p2(pool) * 12;
}

// One CTA's single-count table: 4 counts (class x genotype 0/1) per prefix
// row for each SNP that can follow a (k-2)-prefix (at most n - (k - 2)).
__host__ __device__ inline int64_t pair_sing_words_of(int k, int64_t n)
{
    return n > k - 2 ? (n - (k - 2)) * 4 * (int64_t)ipow3(k - 2) : 0;
}

// next m-subset of [0, n) in lex order whose last element is at most n - 3
// (two SNPs must follow); false after the last
__device__ inline bool next_prefix_pairs(int32_t *p, int m, int64_t n)
{
    const int64_t u = n - 2;
    int t = m - 1;
    while (t >= 0 && p[t] == u - m + t) t--;
    if (t < 0) return false;
    p[t]++;
    for (int v = t + 1; v < m; v++) p[v] = p[v - 1] + 1;
    return true;
}

// the pair of lexicographic index i among the 2-subsets of [c + 1, n)
__device__ __forceinline__ void pair_of_index(int64_t n, int32_t c, int64_t i, int32_t &j1, int32_t &j2)
{
    const int64_t L = n - 1 - c;
    int64_t a = 0, before = 0;
    while (before + (L - 1 - a) <= i) { before += L - 1 - a; a++; }
    j1 = c + 1 + (int32_t)a;
    j2 = j1 + 1 + (int32_t)(i - before);
}

// T(c) = c log2 c of a count below 2^23 with the fast logarithm (0 at c = 0)
__device__ __forceinline__ float tlog_count(uint32_t c)
{
    const float f = u2f_exact(c);
    return f * lg2n(fmaxf(f, 1.0f));
}

// Constants of the screen of the (k-2)-prefix kernel.  With T(c) = c log2 c,
//     m MI / ln 2 = T(m) - T(m1) - T(m0) - sum over cells of
//                   [T(a + b) - T(a) - T(b)]      (a, b: the cell's classes),
// every bracket >= 0 (T is superadditive).  Evaluated with the fast log2 its
// error is bounded by (i) the logarithm: |c (lg2 c - log2 c)| <= 2^-22 (c +
// T(c)) per term, summed over the 27 terms of a row and all rows: at most
// 2^-22 (2 m + mag), mag = T(m) + T(m1) + T(m0) >= the sum of all |terms|
// (superadditivity again); (ii) roundings: the products, a row's chains
// (depth <= 8), the lane's compensated sum, the warp tree (5), the split
// pairs' tree (5) and the final subtraction and scaling: at most 26 u mag.
// The margin doubles that and adds the precise score's own relative bound
// (MI <= ln 2), so every combination whose precise score reaches the
// threshold passes the screen.
struct PairScreen {
    float tconst;        // T(m) - T(m1) - T(m0)
    float ln2_over_m;
    float delta;         // nats
};

__device__ inline PairScreen make_pair_screen(int k, int64_t m, int64_t m1, int64_t m0)
{
    auto T = [](double c) { return c > 0 ? c * log2(c) : 0.0; };
    const double mag = T((double)m) + T((double)m1) + T((double)m0);
    const double u = 5.9604644775390625e-8;
    const double ln2 = 0.6931471805599453;
    PairScreen p;
    p.tconst = (float)(T((double)m) - T((double)m1) - T((double)m0));
    p.ln2_over_m = (float)(ln2 / (double)m);
    p.delta = (float)(2.0 * (2.384185791015625e-7 * (2.0 * (double)m + mag) + 32.0 * u * mag) * ln2 / (double)m +
                      f32_rel_bound(k, m) * ln2) + 1e-7f;
    return p;
}

// Sum of the single-precision MI terms (before the division by m) of
// (prefix, j1, j2) over the prefix rows of blocks part, part + parts, ... of
// 32 kPairRows rows: lanes take rows lane, lane + 32, ... of a block,
// counting per class the joint counts n[g1][g2] (g1, g2 in {0, 1}) over the
// class's word groups; the single counts of the row with j1's and with j2's
// genotype-0/1 rows come from the prefix's single-count table (s1, s2: the
// entries of j1 and j2, [class][genotype][row]).  kScreen: the screen's sum
// of T(a + b) - T(a) - T(b) over the cells instead (PairScreen).  Each lane
// sums compensated, the warp as a tree.
template <int PR, bool kScreen>
__device__ __forceinline__ float score_pair_warp_sum(const uint4 *__restrict__ T, const uint32_t *__restrict__ tot,
                                                     const uint32_t *__restrict__ mj1, const uint32_t *__restrict__ mj2,
                                                     const uint32_t *s1, const uint32_t *s2, int W4, int W14,
                                                     const MiConstF32 &mc, int lane, int part, int parts)
{
    const uint4 *x0p = reinterpret_cast<const uint4 *>(mj1), *x1p = x0p + W4;
    const uint4 *y0p = reinterpret_cast<const uint4 *>(mj2), *y1p = y0p + W4;
    SumF32 acc;
#pragma unroll 1
    for (int r0 = lane + kPairRows * 32 * part; r0 < PR; r0 += kPairRows * 32 * parts) {
        int rr[kPairRows];
#pragma unroll
        for (int i = 0; i < kPairRows; i++) rr[i] = min(r0 + 32 * i, PR - 1);
        // cnt[i][y][q]: q = n00, n01, n10, n11, j1 g0, j1 g1, j2 g0, j2 g1
        uint32_t cnt[kPairRows][2][8];
#pragma unroll
        for (int i = 0; i < kPairRows; i++)
#pragma unroll
            for (int y = 0; y < 2; y++)
#pragma unroll
                for (int q = 0; q < 4; q++) cnt[i][y][q] = 0;
#pragma unroll
        for (int y = 0; y < 2; y++) {
            const int ub = y ? W14 : 0, ue = y ? W4 : W14;
#pragma unroll 1
            for (int u = ub; u < ue; u++) {
                const uint4 x0 = __ldg(x0p + u), x1 = __ldg(x1p + u), y0 = __ldg(y0p + u), y1 = __ldg(y1p + u);
                const uint4 j00 = make_uint4(x0.x & y0.x, x0.y & y0.y, x0.z & y0.z, x0.w & y0.w);
                const uint4 j01 = make_uint4(x0.x & y1.x, x0.y & y1.y, x0.z & y1.z, x0.w & y1.w);
                const uint4 j10 = make_uint4(x1.x & y0.x, x1.y & y0.y, x1.z & y0.z, x1.w & y0.w);
                const uint4 j11 = make_uint4(x1.x & y1.x, x1.y & y1.y, x1.z & y1.z, x1.w & y1.w);
                const size_t off = (size_t)u * PR;
#pragma unroll
                for (int i = 0; i < kPairRows; i++) {
                    const uint4 p = T[off + rr[i]];
                    cnt[i][y][0] += popc4(p, j00);
                    cnt[i][y][1] += popc4(p, j01);
                    cnt[i][y][2] += popc4(p, j10);
                    cnt[i][y][3] += popc4(p, j11);
                }
            }
        }
        // written by this CTA before the barrier that ended the table's
        // build: read through L2 (never the non-coherent path)
#pragma unroll
        for (int i = 0; i < kPairRows; i++)
#pragma unroll
            for (int y = 0; y < 2; y++) {
                cnt[i][y][4] = __ldcg(s1 + (2 * y) * PR + rr[i]);
                cnt[i][y][5] = __ldcg(s1 + (2 * y + 1) * PR + rr[i]);
                cnt[i][y][6] = __ldcg(s2 + (2 * y) * PR + rr[i]);
                cnt[i][y][7] = __ldcg(s2 + (2 * y + 1) * PR + rr[i]);
            }
#pragma unroll
        for (int i = 0; i < kPairRows; i++) {
            if (r0 + 32 * i >= PR) continue;
            uint32_t cell[2][9];
#pragma unroll
            for (int y = 0; y < 2; y++) {
                const uint32_t *c = cnt[i][y];
                const uint32_t t = tot[rr[i] * 2 + y];
                cell[y][0] = c[0];                       // (g1, g2) = (0, 0)
                cell[y][1] = c[1];                       // (0, 1)
                cell[y][2] = c[4] - c[0] - c[1];         // (0, 2)
                cell[y][3] = c[2];                       // (1, 0)
                cell[y][4] = c[3];                       // (1, 1)
                cell[y][5] = c[5] - c[2] - c[3];         // (1, 2)
                cell[y][6] = c[6] - c[0] - c[2];         // (2, 0)
                cell[y][7] = c[7] - c[1] - c[3];         // (2, 1)
                cell[y][8] = t - c[4] - c[5] - cell[y][6] - cell[y][7];   // (2, 2)
            }
            if constexpr (kScreen) {
                float v3[3] = {0.0f, 0.0f, 0.0f};   // three chains of three cells
#pragma unroll
                for (int q = 0; q < 9; q++)
                    v3[q % 3] += tlog_count(cell[0][q] + cell[1][q]) - tlog_count(cell[0][q]) - tlog_count(cell[1][q]);
                acc.add(fmaxf((v3[0] + v3[1]) + v3[2], 0.0f));
            } else {
#pragma unroll
                for (int q = 0; q < 9; q++) acc.add(cell_terms_f32(cell[0][q], cell[1][q], mc));
            }
        }
    }
    float v = acc.value();
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Single-precision MI of (prefix, j1, j2), one warp over all rows.
template <int PR>
__device__ __forceinline__ float score_pair_warp(const uint4 *__restrict__ T, const uint32_t *__restrict__ tot,
                                                 const uint32_t *__restrict__ mj1, const uint32_t *__restrict__ mj2,
                                                 const uint32_t *s1, const uint32_t *s2, int W4, int W14,
                                                 const MiConstF32 &mc, int lane)
{
    return __fdiv_rn(score_pair_warp_sum<PR, false>(T, tot, mj1, mj2, s1, s2, W4, W14, mc, lane, 0, 1), mc.fm);
}

template <int K>
__global__ void __launch_bounds__(kPairThreads, 1) popc_pair_kernel(PopcParams P)
{
    constexpr int km2 = K - 2;
    constexpr int PR = ipow3(K - 2);
    constexpr int PB = PR / 9;
    const PopcDs &D = P.one;
    const DevData d = D.d;
    const int W4 = d.Wt >> 2, W14 = d.W1 >> 2;
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *T = reinterpret_cast<uint4 *>(smem);                          // [W4][PR]
    uint32_t *tot = reinterpret_cast<uint32_t *>(T + (size_t)W4 * PR);   // [PR][2]
    uint64_t *rk = reinterpret_cast<uint64_t *>(smem + ((pair_table_bytes(K, d.Wt) + 15) & ~(size_t)15));
    const int cand_p2 = pair_cand_p2(P.pool);
    float *sc = reinterpret_cast<float *>(rk + cand_p2);
    __shared__ SubtileState S;
    __shared__ int32_t pre[kMaxOrderGpu];
    __shared__ int64_t pbase, i_lo, i_hi;
    __shared__ int32_t jlo;                        // j1 of the CTA's first pair of the prefix
    __shared__ float partial[kPairThreads / 32];   // few pairs: each warp's share of a pair's sum
    __shared__ uint32_t tail_mask;                 // few pairs: those that pass the screen
    // single counts of the prefix rows with the genotype-0/1 rows of each
    // SNP j >= jlo: [j - jlo][class][genotype][row], per CTA in global memory
    uint32_t *sing = P.pair_sing + (size_t)blockIdx.x * (size_t)P.pair_sing_words;
#define EPI_SING_OF(j) (sing + (size_t)((j) - jlo) * 4 * PR)

    const MiConstF32 mc = make_mi_const(d.m, d.m1, d.m0);
    __shared__ PairScreen scr;
    __shared__ int published;                      // the CTA's top_n-th best went out (publish_top_n)
    if (threadIdx.x == 0) {
        scr = make_pair_screen(K, d.m, d.m1, d.m0);
        published = P.top_n <= 0;
    }
    const uint64_t span = D.rank_end - D.rank_begin;
    const uint64_t cb = blockIdx.x - (uint64_t)D.cta_begin, cn = (uint64_t)D.cta_count;
    const int64_t R_b = (int64_t)(D.rank_begin + (uint64_t)(((unsigned __int128)span * cb) / cn));
    const int64_t R_e = (int64_t)(D.rank_begin + (uint64_t)(((unsigned __int128)span * (cb + 1)) / cn));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kPairThreads / 32;

    if (threadIdx.x == 0) {
        S.list_len = 0; S.nbuf = 0; S.thr = -1.0f; S.done = R_b >= R_e;
        if (!S.done) {
            int32_t c[kMaxOrderGpu];
            unrank_lex(d.binom, d.n, K, (uint64_t)R_b, c);
            for (int t = 0; t < km2; t++) pre[t] = c[t];
            // rank of the prefix's first pair (c_last + 1, c_last + 2)
            const int32_t cl = c[km2 - 1];
            const int64_t L = d.n - 1 - cl;
            const int64_t a = c[K - 2] - (cl + 1), b = c[K - 1] - (c[K - 2] + 1);
            const int64_t idx = (a * (2 * L - a - 1)) / 2 + b;
            pbase = R_b - idx;
        }
    }
    __syncthreads();
    while (!S.done) {
        if (threadIdx.x == 0) {
            const int64_t L = d.n - 1 - pre[km2 - 1];
            const int64_t np = L * (L - 1) / 2;
            i_lo = R_b > pbase ? R_b - pbase : 0;
            i_hi = R_e - pbase < np ? R_e - pbase : np;
            if (i_lo < i_hi) {
                int32_t j1, j2;
                pair_of_index(d.n, pre[km2 - 1], i_lo, j1, j2);
                jlo = j1;
            }
            const float g = __uint_as_float(*(volatile uint32_t *)D.global_thr);
            if (S.list_len == P.pool || g > 0.0f) S.thr = fmaxf(S.thr, g);
        }
        __syncthreads();
        // ---- the prefix's table: blocks of 9 rows share the genotypes of
        // the first k-4 SNPs, the last two prefix SNPs give the 9 rows
        for (int idx = threadIdx.x; idx < PB * W4; idx += blockDim.x) {
            const int blk = idx % PB;
            const int w4 = idx / PB;
            uint4 base = make_uint4(~0u, ~0u, ~0u, ~0u);
            int rem = blk, div = PB / 3;
#pragma unroll
            for (int t = 0; t < km2 - 2; t++) {
                const int g = rem / div;
                rem -= g * div;
                div = div > 1 ? div / 3 : 1;
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(d.masks + ((int64_t)pre[t] * 3 + g) * d.Wt) + w4);
                base.x &= v.x; base.y &= v.y; base.z &= v.z; base.w &= v.w;
            }
            const uint4 *ma = reinterpret_cast<const uint4 *>(d.masks + (int64_t)pre[km2 - 2] * 3 * d.Wt);
            const uint4 *mb = reinterpret_cast<const uint4 *>(d.masks + (int64_t)pre[km2 - 1] * 3 * d.Wt);
            uint4 lb[3];
#pragma unroll
            for (int h = 0; h < 3; h++) lb[h] = __ldg(mb + h * W4 + w4);
            uint4 *ps = T + (size_t)w4 * PR + blk * 9;
#pragma unroll
            for (int g = 0; g < 3; g++) {
                const uint4 a = __ldg(ma + g * W4 + w4);
                const uint4 b1 = make_uint4(base.x & a.x, base.y & a.y, base.z & a.z, base.w & a.w);
#pragma unroll
                for (int h = 0; h < 3; h++)
                    ps[g * 3 + h] = make_uint4(b1.x & lb[h].x, b1.y & lb[h].y, b1.z & lb[h].z, b1.w & lb[h].w);
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < PR * 2; idx += blockDim.x) {
            const int row = idx % PR, half = idx / PR;
            const int ub = half ? W14 : 0, ue = half ? W4 : W14;
            uint32_t c = 0;
            for (int u = ub; u < ue; u++) {
                const uint4 v = T[(size_t)u * PR + row];
                c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
            tot[row * 2 + half] = c;
        }
        // the single counts of every SNP that a pair of the CTA's range
        // uses (j1 of its first pair to the last SNP): each serves all
        // the pairs it is part of instead of being counted for each
        if (i_lo < i_hi) {
            const int32_t j0 = jlo;
            const int nj = d.n - j0;
            for (int idx = threadIdx.x; idx < nj * PR * 2; idx += blockDim.x) {
                const int row = idx % PR, rest = idx / PR;
                const int y = rest & 1, jj = rest >> 1;
                const int ub = y ? W14 : 0, ue = y ? W4 : W14;
                const uint4 *g0 = reinterpret_cast<const uint4 *>(d.masks + (int64_t)(j0 + jj) * 3 * d.Wt);
                const uint4 *g1 = g0 + W4;
                uint32_t c0 = 0, c1 = 0;
                for (int u = ub; u < ue; u++) {
                    const uint4 v = T[(size_t)u * PR + row];
                    c0 += popc4(v, __ldg(g0 + u));
                    c1 += popc4(v, __ldg(g1 + u));
                }
                uint32_t *o = sing + ((size_t)jj * 4 + 2 * y) * PR + row;
                __stcg(o, c0);
                __stcg(o + PR, c1);
            }
        }
        __syncthreads();
        // ---- the pairs of this prefix in the CTA's range, in chunks
        const int64_t lo = i_lo, hi = i_hi;
        const int32_t cl = pre[km2 - 1];
        const float thr0 = S.thr;
        // whole rounds of kWarps pairs, one warp per pair; the last q <
        // kWarps pairs (all of them for the prefixes near the end of the SNP
        // order) split each pair's 128-row blocks over kWarps / q warps,
        // whose sums are added as a tree in a fixed order
        const int64_t mid = lo + (hi - lo) / kWarps * kWarps;
        for (int64_t c0 = lo; c0 < mid; c0 += kPairChunk) {
            const int64_t c1 = c0 + kPairChunk < mid ? c0 + kPairChunk : mid;
            const int list_len = S.list_len;
            const float thr = S.thr > thr0 ? S.thr : thr0;
            const float cut = thr - scr.delta;
            for (int64_t i = c0 + warp; i < c1; i += kWarps) {
                int32_t j1, j2;
                pair_of_index(d.n, cl, i, j1, j2);
                // the screen first (warp-uniform; while there is no
                // threshold every pair passes it), the precise score for the
                // pairs within its margin of the threshold
                if (cut > 0.0f) {
                    const float sv = score_pair_warp_sum<PR, true>(
                        T, tot, d.masks + (int64_t)j1 * 3 * d.Wt, d.masks + (int64_t)j2 * 3 * d.Wt, EPI_SING_OF(j1),
                        EPI_SING_OF(j2), W4, W14, mc, lane, 0, 1);
                    if ((scr.tconst - sv) * scr.ln2_over_m < cut) continue;
                }
                const float score = score_pair_warp<PR>(T, tot, d.masks + (int64_t)j1 * 3 * d.Wt,
                                                        d.masks + (int64_t)j2 * 3 * d.Wt, EPI_SING_OF(j1),
                                                        EPI_SING_OF(j2), W4, W14, mc, lane);
                if (lane == 0 && score >= thr) {
                    const int pos = list_len + atomicAdd(&S.nbuf, 1);
                    sc[pos] = score;
                    rk[pos] = (uint64_t)(pbase + i);
                }
            }
            __syncthreads();
            if (S.list_len + S.nbuf + kPairChunk > cand_p2) flush_list(S, sc, rk, P.pool, cand_p2, D.global_thr);
            if (!published && S.list_len + S.nbuf >= P.top_n) {
                publish_top_n(S, sc, rk, P.pool, cand_p2, D.global_thr, P.top_n, K, d.m);
                if (threadIdx.x == 0) published = 1;
                __syncthreads();
            }
        }
        if (mid < hi) {
            const int64_t lo2 = mid;
            const int q = (int)(hi - lo2);
            const int parts = q > 0 ? kWarps / q : 1;
            const int pl = warp / parts, part = warp % parts;
            int32_t j1 = 0, j2 = 0;
            if (pl < q) pair_of_index(d.n, cl, lo2 + pl, j1, j2);
            const uint32_t *m1p = d.masks + (int64_t)j1 * 3 * d.Wt, *m2p = d.masks + (int64_t)j2 * 3 * d.Wt;
            // a pair's sum over its warps' parts, as a tree in a fixed order
            auto tree = [&](int pair) {
                constexpr int kT = kWarps <= 8 ? 8 : (kWarps <= 16 ? 16 : 32);   // a power of two >= kWarps
                float t[kT];
#pragma unroll
                for (int u = 0; u < kT; u++) t[u] = u < parts ? partial[pair * parts + u] : 0.0f;
#pragma unroll
                for (int w2 = kT / 2; w2; w2 >>= 1)
#pragma unroll
                    for (int u = 0; u < w2; u++) t[u] += t[u + w2];
                return t[0];
            };
            // the screen of the q pairs (skipped while there is no
            // threshold), then the precise scores of those within its margin
            // of the threshold (a block-uniform mask)
            const float thr_t = fmaxf(S.thr, thr0);
            float v = 0.0f;
            if (thr_t - scr.delta > 0.0f) {
                if (pl < q)
                    v = score_pair_warp_sum<PR, true>(T, tot, m1p, m2p, EPI_SING_OF(j1), EPI_SING_OF(j2), W4, W14, mc,
                                                      lane, part, parts);
                if (lane == 0) partial[warp] = v;
                if (threadIdx.x == 0) tail_mask = 0;
                __syncthreads();
                if (threadIdx.x < q && (scr.tconst - tree(threadIdx.x)) * scr.ln2_over_m >= thr_t - scr.delta)
                    atomicOr(&tail_mask, 1u << threadIdx.x);
            } else if (threadIdx.x == 0) {
                tail_mask = q >= 32 ? ~0u : (1u << q) - 1u;
            }
            __syncthreads();
            const uint32_t mask = tail_mask;
            if (mask) {
                v = 0.0f;
                if (pl < q && ((mask >> pl) & 1u))
                    v = score_pair_warp_sum<PR, false>(T, tot, m1p, m2p, EPI_SING_OF(j1), EPI_SING_OF(j2), W4, W14, mc,
                                                       lane, part, parts);
                if (lane == 0) partial[warp] = v;
                __syncthreads();
                if (threadIdx.x < q && ((mask >> threadIdx.x) & 1u)) {
                    const float score = __fdiv_rn(tree(threadIdx.x), mc.fm);
                    if (score >= thr_t) {
                        const int pos = S.list_len + atomicAdd(&S.nbuf, 1);
                        sc[pos] = score;
                        rk[pos] = (uint64_t)(pbase + lo2 + threadIdx.x);
                    }
                }
            }
            __syncthreads();
            if (S.list_len + S.nbuf + kPairChunk > cand_p2) flush_list(S, sc, rk, P.pool, cand_p2, D.global_thr);
            if (!published && S.list_len + S.nbuf >= P.top_n) {
                publish_top_n(S, sc, rk, P.pool, cand_p2, D.global_thr, P.top_n, K, d.m);
                if (threadIdx.x == 0) published = 1;
                __syncthreads();
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t L = d.n - 1 - pre[km2 - 1];
            pbase += L * (L - 1) / 2;
            S.done = pbase >= R_e || !next_prefix_pairs(pre, km2, d.n);
        }
        __syncthreads();
    }
    if (S.nbuf > 0) flush_list(S, sc, rk, P.pool, cand_p2, D.global_thr);
    __syncthreads();
    const int Lc = S.list_len;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
        P.list_score[(size_t)blockIdx.x * P.pool + i] = sc[i];
        P.list_rank[(size_t)blockIdx.x * P.pool + i] = rk[i];
    }
    if (threadIdx.x == 0) P.list_count[blockIdx.x] = Lc;
#undef EPI_SING_OF
}

template <int K, int R, bool GP>
static cudaError_t launch_kr(const PopcParams &p, int grid, size_t smem, cudaStream_t st)
{
    auto kern = popc_search_kernel<K, R, GP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, st>>>(p);
    return cudaGetLastError();
}

template <int K, int R, bool GP>
static int occupancy_kr(size_t smem)
{
    auto kern = popc_search_kernel<K, R, GP>;
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 128, smem) != cudaSuccess) return 0;
    return n;
}

// Row-group sizes compiled per order: every R divides 3^(k-1).
bool popc_row_group_ok(int k, int R)
{
    switch (k) {
    case 1: return R == 1;
    case 2: return R == 3;
    case 3: return R == 9;
    case 4: return R == 9 || R == 27;
    case 5: return R == 9 || R == 27;
    case 6: return R == 9;
    case 7: return R == 9;
    case 8: return R == 9;
    default: return false;
    }
}

// orders whose prefix tables may also live in global memory
bool popc_global_prefix_ok(int k, int R) { return (k == 7 || k == 8) && R == 9; }

int popc_default_row_group(int k)
{
    return k == 1 ? 1 : (k == 2 ? 3 : 9);
}

int popc_slot_words(int k, int32_t Wt)
{
    return ipow3(k - 1) * popc_row_stride(k, Wt) + 4;   // 16-byte skew: slots start on different banks
}

size_t popc_smem_bytes(int k, int32_t Wt, int slots, int cand_p2, bool global_prefix)
{
    const size_t PR = (size_t)ipow3(k - 1);
    const size_t pre = global_prefix ? 0 : (size_t)slots * popc_slot_words(k, Wt);
    size_t b = ((pre + (size_t)slots * PR * 2) * 4 + 15) & ~(size_t)15;
    return b + (size_t)cand_p2 * 12;
}

int popc_max_active(int k, int R, size_t smem, bool global_prefix)
{
    if (global_prefix) {
        switch (k * 100 + R) {
        case 709: return occupancy_kr<7, 9, true>(smem);
        case 809: return occupancy_kr<8, 9, true>(smem);
        default: return 0;
        }
    }
    switch (k * 100 + R) {
    case 101: return occupancy_kr<1, 1, false>(smem);
    case 203: return occupancy_kr<2, 3, false>(smem);
    case 309: return occupancy_kr<3, 9, false>(smem);
    case 409: return occupancy_kr<4, 9, false>(smem);
    case 427: return occupancy_kr<4, 27, false>(smem);
    case 509: return occupancy_kr<5, 9, false>(smem);
    case 527: return occupancy_kr<5, 27, false>(smem);
    case 609: return occupancy_kr<6, 9, false>(smem);
    case 709: return occupancy_kr<7, 9, false>(smem);
    case 809: return occupancy_kr<8, 9, false>(smem);
    default: return 0;
    }
}

static cudaError_t launch_dispatch(const PopcParams &p, int k, int R, int grid, size_t smem, cudaStream_t st)
{
    if (p.pre_global) {
        switch (k * 100 + R) {
        case 709: return launch_kr<7, 9, true>(p, grid, smem, st);
        case 809: return launch_kr<8, 9, true>(p, grid, smem, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (k * 100 + R) {
    case 101: return launch_kr<1, 1, false>(p, grid, smem, st);
    case 203: return launch_kr<2, 3, false>(p, grid, smem, st);
    case 309: return launch_kr<3, 9, false>(p, grid, smem, st);
    case 409: return launch_kr<4, 9, false>(p, grid, smem, st);
    case 427: return launch_kr<4, 27, false>(p, grid, smem, st);
    case 509: return launch_kr<5, 9, false>(p, grid, smem, st);
    case 527: return launch_kr<5, 27, false>(p, grid, smem, st);
    case 609: return launch_kr<6, 9, false>(p, grid, smem, st);
    case 709: return launch_kr<7, 9, false>(p, grid, smem, st);
    case 809: return launch_kr<8, 9, false>(p, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

bool popc_pair_applies(int k, int32_t Wt, int pool, bool all_scores)
{
    if (k < EPI_PAIR_MIN_ORDER || k > 8 || all_scores) return false;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    return pair_smem_bytes(k, Wt, pool) <= (size_t)optin;
}

int64_t popc_pair_sing_words(int k, int64_t n) { return pair_sing_words_of(k, n); }

// CTAs of a (k-2)-prefix search: waves of one CTA per SM (tuning parameter:
// equal rank ranges per CTA, so more waves even out prefixes of unequal cost;
// measured on orders 6-8, 2048-4096 samples: 8 waves 6-15 % faster than 1
// and 2-8 % faster than 4, 16 waves another 2-5 %; with the screen 2, 4 and
// 8 waves took 42.2, 38.8 and 34.7 ms at order 8, 23 x 2048), fewer where
// the single-count tables would pass 512 MiB
#ifndef EPI_PAIR_WAVES
#define EPI_PAIR_WAVES 16
#endif
int popc_pair_grid(int num_sms, int k, int64_t n)
{
    const int64_t per_wave = (int64_t)num_sms * pair_sing_words_of(k, n) * 4;
    int64_t waves = per_wave > 0 ? ((int64_t)512 << 20) / per_wave : EPI_PAIR_WAVES;
    waves = waves < 1 ? 1 : (waves > EPI_PAIR_WAVES ? EPI_PAIR_WAVES : waves);
    return num_sms * (int)waves;
}

template <int K>
static cudaError_t launch_pair(const PopcParams &p, int grid, size_t smem, cudaStream_t st)
{
    auto kern = popc_pair_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kPairThreads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_popc_search(const DevData &d, int k, int R, uint64_t rank_begin, uint64_t rank_end, int tile,
                               int pool, int slots, int cand_p2, uint32_t *global_thr, float *list_score,
                               uint64_t *list_rank, int32_t *list_count, int grid, size_t smem, cudaStream_t st,
                               float *all_scores, uint32_t *pre_global, uint32_t *pair_sing, int top_n)
{
    PopcParams p;
    p.top_n = top_n;
    p.all_scores = all_scores;
    p.pre_global = pre_global;
    p.pre_cta_words = (int64_t)slots * popc_slot_words(k, d.Wt);
    p.pair_sing = pair_sing;
    p.pair_sing_words = pair_sing_words_of(k, d.n);
    p.one.d = d;
    p.one.rank_begin = rank_begin;
    p.one.rank_end = rank_end;
    p.one.cta_begin = 0;
    p.one.cta_count = grid;
    p.one.global_thr = global_thr;
    p.many = nullptr;
    p.cta_ds = nullptr;
    p.tile = tile;
    p.pool = pool;
    p.slots = slots;
    p.cand_p2 = cand_p2;
    p.max_wt = d.Wt;
    p.list_score = list_score;
    p.list_rank = list_rank;
    p.list_count = list_count;
    // orders EPI_PAIR_MIN_ORDER-8 with the (k-2)-prefix table in shared
    // memory where it fits and the caller gives the single-count tables
    // (grid x popc_pair_sing_words words); the searches that return every
    // score keep the (k-1)-prefix kernel
    if (pair_sing && popc_pair_applies(k, d.Wt, pool, all_scores != nullptr)) {
        const size_t ps = pair_smem_bytes(k, d.Wt, pool);
        if (k == 6) return launch_pair<6>(p, grid, ps, st);
        return k == 7 ? launch_pair<7>(p, grid, ps, st) : launch_pair<8>(p, grid, ps, st);
    }
    p.pair_sing = nullptr;
    return launch_dispatch(p, k, R, grid, smem, st);
}

size_t popc_ds_bytes() { return sizeof(PopcDs); }

void popc_fill_ds(void *dst, const DevData &d, uint64_t rank_begin, uint64_t rank_end, int cta_begin, int cta_count,
                  uint32_t *global_thr)
{
    PopcDs *o = static_cast<PopcDs *>(dst);
    o->d = d;
    o->rank_begin = rank_begin;
    o->rank_end = rank_end;
    o->cta_begin = cta_begin;
    o->cta_count = cta_count;
    o->global_thr = global_thr;
}

cudaError_t launch_popc_batch(const void *ds_dev, const int32_t *cta_ds_dev, int k, int R, int max_wt, int tile,
                              int pool, int slots, int cand_p2, float *list_score, uint64_t *list_rank,
                              int32_t *list_count, int grid, size_t smem, cudaStream_t st)
{
    PopcParams p;
    p.all_scores = nullptr;
    p.pre_global = nullptr;
    p.pre_cta_words = 0;
    p.pair_sing = nullptr;
    p.pair_sing_words = 0;
    p.top_n = 0;
    p.one = PopcDs();
    p.many = static_cast<const PopcDs *>(ds_dev);
    p.cta_ds = cta_ds_dev;
    p.tile = tile;
    p.pool = pool;
    p.slots = slots;
    p.cand_p2 = cand_p2;
    p.max_wt = max_wt;
    p.list_score = list_score;
    p.list_rank = list_rank;
    p.list_count = list_count;
    return launch_dispatch(p, k, R, grid, smem, st);
}

}  // namespace epi
