// Tensor-core counting path of the exhaustive search (tcgen05, sm_103a).
//
// The last combination level of Section 2.2 (AND of the prefix table with
// the last SNP's table, then popcount) is an exact 0/1 matrix product:
//     count[(p, x'), (j, g)] = sum over individuals s of A[(p, x')][s] * B[(j, g)][s]
// with A[(p, x')] the genotype-table row x' of prefix p (Section 2.1) and
// B[(j, g)] row g of SNP j, summed separately over the case and the control
// individuals.  Both operands hold 0/1 values as FP8 E4M3 bytes and the MMA
// accumulates in FP32 in tensor memory.  Because the product sums over K,
// any fixed permutation of the individuals inside a K stage, applied to both
// operands, leaves the counts unchanged, and the two operands may carry
// different weights per K position as long as their product is constant:
//   * K byte 4 i + b of each 32-individual word holds individual 8 b + i, so
//     the A producer turns one mask word into eight output words with one
//     AND each (output i keeps bit i of every byte, shifted into bits 3..6);
//   * A's nonzero byte at position i is 2^-5, 2^-3, 2^1 or 2^-6 (normal E4M3
//     powers of two) and B's is the reciprocal times 2^-5, so every product
//     of two ones is exactly 2^-5 and an accumulator holds count * 2^-5, an
//     exact FP32 value.
// Genotype 2 of the last SNP is obtained by subtraction from the prefix
// row's total, as in the popcount path.
//
// Layout of one tile: M = 128 rows = 4 warps x 32 lanes; each warp holds
// floor(32 / 3^(k-1)) whole prefixes (prefix rows never straddle a warp, so
// the epilogue reduces a prefix within a warp); N = 128 columns = 64 last
// SNPs x genotypes {0, 1}; K = 128 individuals per stage.  At order 3, where
// the counts fit, the combined-class variant (Shape<true> below) sums both
// classes into one accumulator with E5M2 operands and uses N = 256 columns.
// Prefixes are taken in "panel order" (by their last SNP c ascending) so the
// last SNPs of a tile, j > c, form one contiguous range.  A lexicographic rank
// range [r0, r1) of combinations covers the first SNPs s1 in [a, b] (those of
// ranks r0 and r1 - 1); within a panel the prefixes are listed
// lexicographically, so the ones with s1 in [a, b] are contiguous, and the
// epilogue keeps, per prefix, only the last SNPs whose combination's rank lies
// in [r0, r1) (consecutive ranks share their prefix and differ in the last
// SNP, so that is one interval of j).
//
// Warp roles (by default 576 threads = 18 warps, one CTA per SM, persistent,
// a contiguous range of work items per CTA; an item = one M tile x one N
// tile x the whole K range; the epilogue/producer split is Roles<C, K>
// below: 8/8, or 12/4 for the combined-class variant):
//   epilogue warps (first): TMEM -> registers, single-precision MI screen,
//               exact-margin candidate selection, per-CTA candidate list;
//               warp w reads TMEM lane quadrant w % 4 for the chunks of 8
//               last SNPs w / 4, w / 4 + G, ... (G warps per quadrant)
//   A producers: prefix rows = AND of the prefix SNPs' bit rows, expanded
//               to FP8 bytes in the 128-byte-swizzled K-major layout; one
//               thread per row, groups of 4 warps taking the ring's stages
//               in turn, own stages prefetched
//   next warp   TMA producer of B tiles, and writer of the item descriptors
//   last warp   TMEM allocator and MMA issuer (one elected thread)
// Every mbarrier wait is bounded (about 2 s); a wait that gives up sets
// ST_TIMEOUT and all roles leave their loops, drain their own asynchronous
// work and free tensor memory.
#include <cuda.h>
#include <cstring>
#include <cudaTypedefs.h>

#include "epi_host.h"
#include "epi_internal.cuh"
#include "epi_tcgen05.cuh"

// A producers' load distance in K stages (tuning parameter); the
// stage-release group size is chosen per order (EPI_TC_RELEASE overrides it)
#ifndef EPI_TC_PREFETCH
#define EPI_TC_PREFETCH 2
#endif

namespace epi {

namespace tc {

constexpr int kKC = 128;               // individuals (bytes) per K stage

// Tile shapes of the two variants.
//   separate classes (C = false): N tile = 64 last SNPs (128 columns), E4M3
//     operands, one accumulator per class (2 x 128 columns, double buffered),
//     6 stages of A and B tiles;
//   combined classes (C = true): N tile = 128 last SNPs (256 columns), E5M2
//     operands whose case products are 2^p times the control products, so
//     one accumulator holds ctrl + case * 2^p (exact while below 2^23);
//     double buffered in 2 x 256 columns; 4 stages of A (128 rows) and B
//     (256 rows) tiles.  The MMA of an N tile that ends the last SNPs is cut
//     to the columns in use (a multiple of 16).
template <bool C>
struct Shape {
    static constexpr int J = C ? 128 : 64;          // last SNPs per N tile
    static constexpr int N = 2 * J;                 // tile columns
    static constexpr int Stages = C ? 4 : 6;        // K stages in the rings
    static constexpr int BBytes = N * kKC;          // one B stage
};

// Epilogue warps of the separate-class variant at order 4 (tuning
// parameter; the other 16 - n warps produce A tiles).  Measured: 8 (two
// producer groups) 126.5 ms at 300 SNPs x 4000 and 1522 ms at 500 x 8192;
// 4 (three producer groups) 190 and 1579 ms.
#ifndef EPI_TC_K4_EPI_WARPS
#define EPI_TC_K4_EPI_WARPS 8
#endif

// Warp roles of an order-K launch.  The combined variant's producers write
// each A row once per 512-cycle stage, so one group of 4 warps keeps up and
// 12 warps (3 per TMEM lane quadrant) run the epilogue; the separate variant
// has producer groups of 4 warps taking the ring's stages in turn.
// Epilogue and producer warps of the combined-class variant (tuning
// parameters; the launch's register cap follows from the warps per SM
// sub-partition.  Order 3, 2000 x 4000: 12 + 4 warps (96 registers) 86.6 ms,
// 8 + 4 (128 registers) 88.3 ms, 8 + 8 93.6 ms, 12 + 8 (80 registers,
// spills) 100.6 ms; before the screen's logarithms lost their subnormal
// handling: 93.8, 100.1, 110.8 ms, and 4 + 4 133.5 ms)
#ifndef EPI_TC_C_EPI_WARPS
#define EPI_TC_C_EPI_WARPS 12
#endif
#ifndef EPI_TC_C_PROD_WARPS
#define EPI_TC_C_PROD_WARPS 4
#endif

template <bool C, int K>
struct Roles {
    static constexpr int J = Shape<C>::J;
    static constexpr int EpiWarps = C ? EPI_TC_C_EPI_WARPS : (K == 4 ? EPI_TC_K4_EPI_WARPS : 8);
    static constexpr int ProdWarps = C ? EPI_TC_C_PROD_WARPS : 16 - EpiWarps;
    static constexpr int Threads = 32 * (EpiWarps + ProdWarps + 2);   // + the TMA and MMA warps
    static constexpr int EpiThreads = 32 * EpiWarps;
    static constexpr int ProdGroups = ProdWarps / 4;  // one thread per tile row each
    static constexpr int ColGroups = EpiWarps / 4;    // epilogue warps per lane quadrant
    // chunks of 8 last SNPs per epilogue warp and item, and the chunks
    // between two candidate-buffer checks (a barrier of the epilogue warps
    // and maybe a sort): every 2 chunks with separate classes, once per item
    // with combined classes (its larger buffer then lives in global memory)
    static constexpr int Iters = (J / 8 + ColGroups - 1) / ColGroups;
    static constexpr int CheckIters = C ? Iters : 2;
    static_assert(EpiWarps % 4 == 0 && ProdWarps % 4 == 0, "roles come in whole lane quadrants");
};
constexpr int kMaxProdGroups = 3;

// the host's view of the roles of a launch (order k, variant comb)
inline int roles_epi_warps(bool comb, int k)
{
    return comb ? Roles<true, 3>::EpiWarps : (k == 4 ? Roles<false, 4>::EpiWarps : Roles<false, 3>::EpiWarps);
}
inline int roles_check_iters(bool comb, int k)
{
    return comb ? Roles<true, 3>::CheckIters : (k == 4 ? Roles<false, 4>::CheckIters : Roles<false, 3>::CheckIters);
}
// Stages are released to the producers in groups: a tcgen05.commit lets the
// following MMAs start only after the earlier ones finish (about one MMA
// latency of idle tensor pipe), so the issuer commits once per group of
// kRelease stages instead of once per stage.
// measured best: groups of 2 stages at orders 2-3 (the epilogue bounds the
// issuer), single stages at orders 4-5 (the A producers do)
template <int K, bool C>
constexpr int release_group()
{
#ifdef EPI_TC_RELEASE
    return EPI_TC_RELEASE;
#else
    return C ? 1 : (K <= 3 ? 2 : 1);
#endif
}
constexpr int kDescDepth = 4;
static_assert(Roles<false, 4>::ProdWarps / 4 <= 3, "at most kMaxProdGroups producer groups");
constexpr int kTileBytes = 128 * kKC;        // one A tile (and a B tile of the separate-class variant)
constexpr int kWaitSlots = 8;
constexpr int kMaxDescSnps = 40;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

struct Desc {
    int32_t j0;          // first last-SNP of the N tile
    int32_t nvalid;      // real prefixes in the M tile
    int32_t snp[kMaxDescSnps];   // prefix p occupies snp[p*(k-1) .. p*(k-1)+k-2]
};

// One dataset of a launch; a batched launch covers several datasets of the
// same order, CTAs [cta_begin, cta_begin + cta_count) working on this one.
struct DsParams {
    DevData d;
    uint64_t n_prefix;         // prefixes searched (first SNP in [s1_lo, s1_hi])
    uint64_t n_items;
    const uint64_t *item_cum;  // [n + 1] items of M tiles starting in panels < c
    const uint64_t *pcum;      // [n + 1] prefixes searched in panels < c
    uint64_t rank_begin, rank_end;   // lexicographic ranks searched
    int32_t s1_lo, s1_hi;      // first SNPs of ranks rank_begin and rank_end - 1
    int32_t clip;              // 0: the whole combination range
    int32_t comb_p;            // combined-class variant: control counts in the low comb_p bits
    int chunks, chunks_case;   // K stages in total / over the cases
    float delta;               // screening margin (nats)
    float tconst;              // T(m) - T(m1) - T(m0), T(c) = c log2 c
    float ln2_over_m;
    uint64_t total;            // C(n, k)
    uint32_t *global_thr;
    const CUtensorMap *tmap;   // B-operand map in global memory (batched launches)
    int32_t cta_begin, cta_count;
};

struct Params {
    DsParams one;              // the dataset when the launch has one
    const DsParams *many;      // else [n_ds] in device memory
    const int32_t *cta_ds;     // and the dataset of each CTA
    int k, PR, ppw, ppt;
    int pool, cand_p2;
    // the CTA's candidate buffer [cand_p2] in global memory (per CTA, at
    // blockIdx.x * cand_p2) where it does not fit in shared memory; NULL:
    // shared memory
    float *cand_score_g;
    uint64_t *cand_rank_g;
    float *list_score;
    uint64_t *list_rank;
    int32_t *list_count;
    int32_t *status;
    unsigned long long wait_ns;   // limit of the pipeline waits (0: kTimeoutNs)
    uint32_t *dump;            // optional: every table, [rank][2][3^k] (validation)
    unsigned long long *waits; // optional: [grid][8] cycles spent waiting, per role (tracing)
};

// ------------------------------------------------------------------ PTX --
// Limit of the pipeline waits of this CTA (set at start from Params.wait_ns,
// the default kTimeoutNs when 0).  The drain waits at exit always use
// kTimeoutNs, so that no asynchronous copy or MMA is outstanding when the CTA
// leaves.
__shared__ unsigned long long g_wait_limit_ns;

// Bounded wait for the phase of parity `parity`; false when it gave up (the
// CTA-wide abort flag is then set).
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    const unsigned long long limit = g_wait_limit_ns;
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (now_ns() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
    }
}

// Hot-path wait: one inline non-blocking test; the bounded out-of-line wait
// (and the cycle accounting of the trace) only when the phase is not
// complete yet, so the trace counts every cycle spent waiting.
__device__ __forceinline__ bool wait_fast(uint64_t *bar, uint32_t parity, volatile int *abort_flag, long long &acc)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    const bool ok = mbar_wait(bar, parity, abort_flag);
    acc += clock64() - t0;
    return ok;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Instruction descriptor of kind::f8f6f4 with F32 accumulation, K-major A
// and B, M = 128 and n columns; operand format 0 = E4M3, 1 = E5M2 (both).
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t n)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdesc = make_idesc(0, 128);

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

// The same MMA executed by a whole warp in step; only the elected lane
// (`leader` nonzero) issues it.
__device__ __forceinline__ void mma_f8_warp(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                            uint32_t leader, uint32_t idesc = kIdesc)
{
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 e, %5, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate), "r"(leader));
}

__device__ __forceinline__ void mma_commit_warp(uint64_t *bar, uint32_t leader)
{
    asm volatile(
        "{\n .reg .pred e;\n setp.ne.b32 e, %1, 0;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(smem_u32(bar)),
        "r"(leader)
        : "memory");
}

__device__ __forceinline__ uint32_t elect_one()
{
    uint32_t pred;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
    return pred;
}

template <int NT>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// ------------------------------------------------------------ enumeration --
// Prefixes of order k are the (k-1)-subsets whose last SNP c is <= n-2, in
// panel order: panel c holds the subsets ending in c whose first SNP lies in
// [s1_lo, s1_hi], their first k-2 SNPs in lexicographic order.  pcum[c]
// counts the prefixes of panels < c; q is a prefix's index in this order.
struct PrefixIter {
    int32_t a[kMaxOrderTc];    // first k-2 SNPs (ascending)
    int32_t c;                 // last prefix SNP (panel)
    uint64_t q;                // index in panel order
};

// Subsets of [0, c) of size m with first element >= x: C(c - x, m) (0 when
// c - x < m); for m = 0 the single empty subset, which has no first element
// and counts for every x.
__device__ __forceinline__ uint64_t subsets_from(const DevData &d, int64_t c, int64_t x, int m)
{
    if (m == 0) return 1;
    return c - x >= m ? binom_at(d.binom, d.n, c - x, m) : 0;
}

// Lexicographic unranking of r among the m-subsets of [0, c) (m <= 3).
__device__ inline void lex_unrank_below(const DevData &d, int64_t c, int m, uint64_t r, int32_t *out)
{
    int64_t start = 0;
    for (int i = 0; i < m; i++) {
        const int rem = m - i;
        const uint64_t all = binom_at(d.binom, d.n, c - start, rem);
        // largest x in [start, c - rem] with fewer than r + 1 subsets whose
        // element i is below x
        int64_t lo = start, hi = c - rem;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (all - binom_at(d.binom, d.n, c - mid, rem) <= r) lo = mid;
            else hi = mid - 1;
        }
        r -= all - binom_at(d.binom, d.n, c - lo, rem);
        out[i] = (int32_t)lo;
        start = lo + 1;
    }
}

__device__ inline void prefix_unrank(const DsParams &P, int k, uint64_t q, PrefixIter &it)
{
    const DevData &d = P.d;
    // panel: largest c with pcum[c] <= q (a non-empty panel)
    int64_t lo = 0, hi = d.n - 2;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (P.pcum[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    it.c = (int32_t)lo;
    it.q = q;
    const int m2 = k - 2;
    // index within the panel: the subsets whose first SNP is below s1_lo come first
    const uint64_t skip = subsets_from(d, lo, 0, m2) - subsets_from(d, lo, P.s1_lo, m2);
    lex_unrank_below(d, lo, m2, (m2 ? skip : 0) + (q - P.pcum[lo]), it.a);
}

__device__ inline void prefix_next(const DsParams &P, int k, PrefixIter &it)
{
    it.q++;
    const int m2 = k - 2;
    // lexicographic successor within the panel: the last position that can
    // still grow; the first SNP must stay <= s1_hi
    int i = m2 - 1;
    while (i >= 0 && it.a[i] >= it.c - m2 + i) i--;
    if (i > 0 || (i == 0 && it.a[0] + 1 <= P.s1_hi)) {
        it.a[i]++;
        for (int t = i + 1; t < m2; t++) it.a[t] = it.a[t - 1] + 1;
        return;
    }
    // next panel (every panel after a non-empty one is non-empty): its first
    // prefix starts at s1_lo
    it.c++;
    for (int t = 0; t < m2; t++) it.a[t] = P.s1_lo + t;
}

template <int J>
__device__ __forceinline__ int64_t ntiles_of(const DevData &d, int32_t c) { return (d.n - 1 - c + J - 1) / J; }

// -------------------------------------------------------------- epilogue --
// accumulator = count * 2^-5 (exact): the count as a float, and as an integer
__device__ __forceinline__ uint32_t f2u_exact(float v) { return __float_as_uint(v + 8388608.0f) & 0x7FFFFFu; }

// Combined-class accumulator x = 2^-12 (ctrl + case 2^p), an integer v
// below 2^23 times 2^-12: y = fma(x, 2^12, 2^23) = 2^23 + v holds v in its
// 23 mantissa bits (exact).  Keeping the low p bits under the exponent of
// 2^23 gives 2^23 + ctrl, hence ctrl / 32 in one fused multiply-add, and
// y - (2^23 + ctrl) = case 2^p exactly, hence case / 32 in one multiply by
// case_scale = 2^-(p+5).  Both come out as the separate-class variant's
// accumulator values (count / 32).
__device__ __forceinline__ void split_classes(uint32_t x, uint32_t lo_mask, float case_scale, uint32_t &case32,
                                              uint32_t &ctrl32)
{
    const float y = fmaf(__uint_as_float(x), 4096.0f, 8388608.0f);
    const float lo = __uint_as_float((__float_as_uint(y) & lo_mask) | 0x4B000000u);
    ctrl32 = __float_as_uint(fmaf(lo, 0.03125f, -262144.0f));
    case32 = __float_as_uint((y - lo) * case_scale);
}

// t(x) = x log2 x of an accumulator value x = count / 32 (0 for x = 0)
__device__ __forceinline__ float tlog32(float x) { return x * lg2n(fmaxf(x, 0.03125f)); }

// sum over the three cells of one tile row of t(a) + t(b) - t(a + b) (a, b:
// case and control accumulators): one fused multiply-add chain per cell,
// the three cells side by side, then two adds
__device__ __forceinline__ float row_screen(float a0, float a1, float a2, float b0, float b1, float b2)
{
    const float s0 = a0 + b0, s1 = a1 + b1, s2 = a2 + b2;
    float v0 = a0 * lg2n(fmaxf(a0, 0.03125f));
    float v1 = a1 * lg2n(fmaxf(a1, 0.03125f));
    float v2 = a2 * lg2n(fmaxf(a2, 0.03125f));
    v0 = fmaf(b0, lg2n(fmaxf(b0, 0.03125f)), v0);
    v1 = fmaf(b1, lg2n(fmaxf(b1, 0.03125f)), v1);
    v2 = fmaf(b2, lg2n(fmaxf(b2, 0.03125f)), v2);
    v0 = fmaf(-s0, lg2n(fmaxf(s0, 0.03125f)), v0);
    v1 = fmaf(-s1, lg2n(fmaxf(s1, 0.03125f)), v1);
    v2 = fmaf(-s2, lg2n(fmaxf(s2, 0.03125f)), v2);
    return (v0 + v1) + v2;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int PR>
__device__ __forceinline__ float seg_sum(float v, int pos)
{
#pragma unroll
    for (int off = 1; off < PR; off <<= 1) {
        const float o = __shfl_down_sync(0xffffffffu, v, off);
        if ((pos & (2 * off - 1)) == 0 && pos + off < PR) v += o;
    }
    return v;
}

template <int NT>
__device__ inline void sort_cands_epi(float *sc, uint64_t *rk, int p2, int tid)
{
    for (int kk = 2; kk <= p2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = tid; i < p2; i += NT) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const bool sw = up ? cand_better(sc[ixj], rk[ixj], sc[i], rk[i])
                                       : cand_better(sc[i], rk[i], sc[ixj], rk[ixj]);
                    if (sw) {
                        float ts = sc[i]; sc[i] = sc[ixj]; sc[ixj] = ts;
                        uint64_t tr = rk[i]; rk[i] = rk[ixj]; rk[ixj] = tr;
                    }
                }
            }
            epi_bar<NT>();
        }
    }
}

struct EpiState {
    int32_t list_len, nbuf, stop;
    float thr;
};

template <int NT>
__device__ inline void epi_flush(EpiState &S, float *sc, uint64_t *rk, int pool, uint32_t *global_thr, int tid)
{
    epi_bar<NT>();
    const int live = S.list_len + S.nbuf;
    const int p2 = next_pow2(live < 2 ? 2 : live);
    for (int i = live + tid; i < p2; i += NT) { sc[i] = -1.0f; rk[i] = ~0ull; }
    epi_bar<NT>();
    sort_cands_epi<NT>(sc, rk, p2, tid);
    if (tid == 0) {
        S.list_len = live < pool ? live : pool;
        S.nbuf = 0;
        if (S.list_len == pool) {
            S.thr = sc[pool - 1];
            atomicMax(global_thr, __float_as_uint(S.thr));
        }
    }
    epi_bar<NT>();
}

// ---------------------------------------------------------------- kernel --
// Precise single-precision terms of one tile row's three cells (the rare
// candidate path, kept out of line).
__device__ __noinline__ float row_terms_precise(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, uint32_t a2,
                                                uint32_t b2, const MiConstF32 mc)
{
    return cell_terms_f32(a0, b0, mc) + cell_terms_f32(a1, b1, mc) + cell_terms_f32(a2, b2, mc);
}

#define TMEM_LD16(taddr, r)                                                                                      \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
                 "[%16];"                                                                                        \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),       \
                   "=r"(r[15])                                                                                   \
                 : "r"(taddr))

template <int K, bool C>
__global__ void __launch_bounds__(Roles<C, K>::Threads, 1) tc_search_kernel(const __grid_constant__ CUtensorMap tmap_b,
                                                                const Params P)
{
    static_assert(!C || K == 3, "the combined-class variant serves order 3");
    using S = Shape<C>;
    using R = Roles<C, K>;
    constexpr int kStages = S::Stages;
    constexpr int kJ = S::J;
    constexpr int kBBytes = S::BBytes;
    constexpr int kEpiWarps = R::EpiWarps, kProdWarps = R::ProdWarps, kEpiThreads = R::EpiThreads;
    constexpr int kGroups = R::ProdGroups, kCG = R::ColGroups;
    // epilogue: the kQC chunks of 8 last SNPs of a lane quadrant go round-
    // robin to its kCG warps, kIters chunks each (the last may be empty)
    constexpr int kQC = kJ / 8;
    constexpr int kIters = R::Iters;
    constexpr int kPR = K == 2 ? 3 : (K == 3 ? 9 : (K == 4 ? 27 : 81));
    // order 5: one prefix per tile, its 81 rows over lane quadrants 0-2 (the
    // epilogue sums a combination across warps through shared memory)
    constexpr bool kWide = kPR > 32;
    constexpr int kPPW = kWide ? 0 : 32 / kPR;
    constexpr int kPPT = kWide ? 1 : 4 * kPPW;
    constexpr int km1 = K - 1;
    constexpr int kWarpTma = kEpiWarps + kProdWarps;
    constexpr int kWarpMma = kWarpTma + 1;
    // candidate-buffer checks (a barrier and maybe a sort) every kJcPerCheck
    // chunks of 8 last SNPs; the buffer holds the pool and one interval
    constexpr int kJcPerCheck = K == 2 ? 1 : R::CheckIters;
    static_assert(kIters % kJcPerCheck == 0, "every item ends on a candidate-buffer check");
    constexpr int kRelease = release_group<K, C>();
    // orders 3-4: prefix sums through the shared transpose buffer
    constexpr bool kTranspose = K == 3 || K == 4;
    constexpr int kPairs = kWide ? 0 : kPPW * 8;              // (prefix, last SNP) pairs per warp and chunk
    constexpr int kPairIters = (kPairs + 31) / 32;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char *stages_a = smem;
    unsigned char *stages_b = smem + kStages * kTileBytes;
    float *sc;
    uint64_t *rk;
    uint32_t *tot;                               // [2][128][kMaxProdGroups][2 classes]
    if (P.cand_score_g) {
        sc = P.cand_score_g + (size_t)blockIdx.x * P.cand_p2;
        rk = P.cand_rank_g + (size_t)blockIdx.x * P.cand_p2;
        tot = reinterpret_cast<uint32_t *>(stages_b + kStages * kBBytes);
    } else {
        sc = reinterpret_cast<float *>(stages_b + kStages * kBBytes);
        rk = reinterpret_cast<uint64_t *>(sc + P.cand_p2);
        tot = reinterpret_cast<uint32_t *>(rk + P.cand_p2);
    }
    Desc *desc = reinterpret_cast<Desc *>(tot + 2 * 128 * kMaxProdGroups * 2);
    // orders 3-4: per epilogue warp, the row terms of 8 last SNPs [lane][8]
    // (transposed so that one lane sums one prefix's rows for one last SNP)
    unsigned char *after_desc = reinterpret_cast<unsigned char *>(desc + kDescDepth);
    float *wsum = reinterpret_cast<float *>(after_desc + ((16 - (smem_u32(after_desc) & 15)) & 15));

    // one "stage free" barrier per stage for both operands (the A and B rings
    // advance together), released by one MMA commit
    static_assert(kStages % kRelease == 0, "release groups tile the ring");
    static_assert(kStages % kGroups == 0, "each producer group takes every kGroups-th ring slot");
    // full_ab[s]: the A producer warps of the slot's parity and the TMA
    // thread (with its bytes) have filled stage s of both operands
    __shared__ __align__(8) uint64_t full_ab[kStages], empty_ab[kStages / kRelease];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], tot_full[2];
    __shared__ __align__(8) uint64_t desc_full[kDescDepth], desc_empty[kDescDepth], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    // combined variant: the MMA instruction descriptor of each item (its
    // column count), written with the item's descriptor
    __shared__ uint32_t item_idesc[kDescDepth];
    __shared__ volatile int abort_flag;
    __shared__ EpiState ES;
    // order 5: per-warp partial sums [jhalf][quadrant][last SNP of the chunk]
    __shared__ float wred[2][4][8], wpre[2][4][8];
    __shared__ int wflag[2][8];

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const DsParams &DS = P.many ? P.many[P.cta_ds[blockIdx.x]] : P.one;
    const DevData d = DS.d;
    const CUtensorMap *tmap = DS.tmap ? DS.tmap : &tmap_b;

    const uint64_t cb = blockIdx.x - (uint64_t)DS.cta_begin, cn = (uint64_t)DS.cta_count;
    const uint64_t it_b = (uint64_t)(((unsigned __int128)DS.n_items * cb) / cn);
    const uint64_t it_e = (uint64_t)(((unsigned __int128)DS.n_items * (cb + 1)) / cn);
    const int64_t n_my = (int64_t)(it_e - it_b);

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full_ab[s], kProdWarps / kGroups + 1);   // one producer group + the TMA thread
            if (s % kRelease == 0) mbar_init(&empty_ab[s / kRelease], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);
            mbar_init(&tot_full[b], kProdWarps);
        }
        for (int q = 0; q < kDescDepth; q++) {
            mbar_init(&desc_full[q], 1);
            mbar_init(&desc_empty[q], kEpiWarps + kProdWarps);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        g_wait_limit_ns = P.wait_ns ? P.wait_ns : kTimeoutNs;
        ES.list_len = 0; ES.nbuf = 0; ES.stop = 0; ES.thr = -1.0f;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWarpMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == kWarpTma) {
        // ------------------------------------------------ TMA + descriptors
        if (lane == 0 && n_my > 0) {
            const uint64_t w0 = it_b;
            int64_t lo = 0, hi = d.n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (DS.item_cum[mid] <= w0) lo = mid;
                else hi = mid - 1;
            }
            const int32_t c0 = (int32_t)lo;
            const uint64_t off = w0 - DS.item_cum[c0];
            const int64_t nt0 = ntiles_of<kJ>(d, c0);
            const uint64_t tfirst = (DS.pcum[c0] + kPPT - 1) / kPPT;
            const uint64_t t = tfirst + off / (uint64_t)nt0;
            int64_t u = (int64_t)(off % (uint64_t)nt0);
            PrefixIter it;
            prefix_unrank(DS, K, t * (uint64_t)kPPT, it);
            int32_t tile_snp[kPPT * km1];
            int32_t nvalid = 0, cmin = it.c;
            auto fill_tile = [&]() {
                nvalid = 0;
                cmin = it.c;
#pragma unroll
                for (int p = 0; p < kPPT; p++) {
                    if (it.q < DS.n_prefix) {
#pragma unroll
                        for (int s2 = 0; s2 < km1 - 1; s2++) tile_snp[p * km1 + s2] = it.a[s2];
                        tile_snp[p * km1 + km1 - 1] = it.c;
                        nvalid++;
                        prefix_next(DS, K, it);
                    }
                }
            };
            fill_tile();
            uint64_t g = 0;
            long long w_tma = 0;
            for (int64_t i = 0; i < n_my && !abort_flag; i++) {
                const int dq = (int)(i % kDescDepth);
                const uint32_t ud = (uint32_t)(i / kDescDepth);
                if (!mbar_wait(&desc_empty[dq], (ud & 1) ^ 1, &abort_flag)) break;
                Desc &D = desc[dq];
                D.j0 = cmin + 1 + (int32_t)(u * kJ);
                D.nvalid = nvalid;
#pragma unroll
                for (int q = 0; q < kPPT * km1; q++) D.snp[q] = tile_snp[q];
                if constexpr (C) {
                    // columns in use: 2 per last SNP below n, in steps of 16
                    const int32_t live = 2 * ((int32_t)d.n - D.j0);
                    const uint32_t ncol = live >= S::N ? (uint32_t)S::N : (uint32_t)((live + 15) & ~15);
                    item_idesc[dq] = make_idesc(1, ncol);
                }
                mbar_arrive(&desc_full[dq]);
                const int y = 2 * D.j0;
                for (int kc = 0; kc < DS.chunks; kc++, g++) {
                    const int s = (int)(g % kStages);
                    const uint32_t us = (uint32_t)(g / kStages);
                    if (!wait_fast(&empty_ab[s / kRelease], (us & 1) ^ 1, &abort_flag, w_tma)) break;
                    mbar_arrive_tx(&full_ab[s], (uint32_t)kBBytes);
                    tma_load_2d(stages_b + s * kBBytes, tmap, kc * kKC, y, &full_ab[s]);
                }
                u++;
                if (u == ntiles_of<kJ>(d, cmin)) {
                    u = 0;
                    fill_tile();
                }
            }
            if (P.waits) P.waits[blockIdx.x * kWaitSlots + 6] = (unsigned long long)w_tma;
            for (int s = 0; s < kStages; s++) {
                if (g > (uint64_t)s) {
                    const uint64_t last = ((g - 1 - s) / kStages) * kStages + s;
                    const uint32_t us = (uint32_t)(last / kStages);
                    const uint64_t t0 = now_ns();
                    while (!mbar_try(&full_ab[s], us & 1) && now_ns() - t0 < kTimeoutNs) {}
                }
            }
        }
    } else if (warp == kWarpMma) {
        // ------------------------------------------------------------- MMA
        if (n_my > 0) {
            // a lean issue loop run by the whole warp in step (warp-uniform
            // values stay on the uniform datapath); one elected lane issues
            // the MMAs and commits.  The tensor pipe is fed only as fast as
            // this instruction stream runs, so stage descriptors are formed
            // by one add and the ring position and phase are carried.
            const uint32_t leader = elect_one();
            const uint64_t ad0 = sdesc(smem_u32(stages_a)), bd0 = sdesc(smem_u32(stages_b));
            // stage strides in descriptor address units
            constexpr uint32_t kStageDescA = kTileBytes >> 4, kStageDescB = kBBytes >> 4;
            int s = 0;
            uint32_t ph = 0;
            const int chunks = DS.chunks, chunks_case = DS.chunks_case;
            long long w_a = 0, w_b = 0, w_acc = 0;
            const long long t_start = clock64();
            for (int64_t i = 0; i < n_my && !abort_flag; i++) {
                const int b = (int)(i & 1);
                const uint32_t ub = (uint32_t)(i >> 1);
                if (!wait_fast(&acc_empty[b], (ub & 1) ^ 1, &abort_flag, w_acc)) break;
                tc_fence_after();
                // separate classes: case and control accumulators of 128
                // columns each; combined: one accumulator of 256 columns
                const uint32_t d_case = tmem_base + (uint32_t)(b * 256), d_ctrl = d_case + (C ? 0u : 128u);
                uint32_t idesc = kIdesc;
                bool ok = true;
                for (int kc = 0; kc < chunks; kc++) {
                    if (!wait_fast(&full_ab[s], ph, &abort_flag, w_a)) { ok = false; break; }
                    tc_fence_after();
                    // the item's column count is in place once its first stage is full
                    if (C && kc == 0) idesc = item_idesc[i % kDescDepth];
                    const uint32_t dcol = kc < chunks_case ? d_case : d_ctrl;
                    const uint32_t acc0 = (kc == 0 || (!C && kc == chunks_case)) ? 0u : 1u;
                    const uint64_t ad = ad0 + (uint64_t)(s * kStageDescA), bd = bd0 + (uint64_t)(s * kStageDescB);
                    mma_f8_warp(dcol, ad, bd, acc0, leader, idesc);
#pragma unroll
                    for (int kk = 1; kk < kKC / 32; kk++)
                        mma_f8_warp(dcol, ad + 2 * kk, bd + 2 * kk, 1u, leader, idesc);
                    if (s % kRelease == kRelease - 1) mma_commit_warp(&empty_ab[s / kRelease], leader);
                    if (++s == kStages) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                mma_commit_warp(&acc_full[b], leader);
            }
            if (P.waits && leader) {
                unsigned long long *wp = P.waits + blockIdx.x * kWaitSlots;
                wp[0] = (unsigned long long)w_a;
                wp[1] = (unsigned long long)w_b;
                wp[2] = (unsigned long long)w_acc;
                wp[7] = (unsigned long long)(clock64() - t_start);
            }
            __syncwarp();
            mma_commit_warp(&drain_bar, leader);
            const uint64_t t0 = now_ns();
            while (!mbar_try(&drain_bar, 0) && now_ns() - t0 < kTimeoutNs) {}
        }
    } else if (warp >= kEpiWarps) {
        // ---------------------------------------------------- A producers
        // Thread t owns tile row r = t % 128 in the ring slots of group
        // t / 128 (with two groups they take alternate stages), and writes
        // all 128 individuals of the row's stage: four mask words, each
        // expanded to 32 bytes.
        const int t = tid - kEpiThreads;     // 0 .. 32 kProdWarps - 1
        const int r = t & 127;
        const int grp = t >> 7;
        const int l = r & 31, w = r >> 5;
        uint64_t g = 0;                      // stages of the CTA so far (both halves)
        long long w_prod = 0, w_prod_acc = 0;
        for (int64_t i = 0; i < n_my; i++) {
            if (abort_flag) break;
            const int dq = (int)(i % kDescDepth);
            const uint32_t ud = (uint32_t)(i / kDescDepth);
            if (!mbar_wait(&desc_full[dq], ud & 1, &abort_flag)) break;
            const Desc &D = desc[dq];
            const uint4 *rows[km1];
            bool active = false;
            if (kWide ? r < kPR : l < kPPW * kPR) {
                const int p = kWide ? 0 : w * kPPW + l / kPR;
                if (p < D.nvalid) {
                    active = true;
                    int rem = kWide ? r : l % kPR, div = kPR / 3;
#pragma unroll
                    for (int tt = 0; tt < km1; tt++) {
                        const int gg = rem / div;
                        rem -= gg * div;
                        div = div > 1 ? div / 3 : 1;
                        rows[tt] = reinterpret_cast<const uint4 *>(d.masks + ((int64_t)D.snp[p * km1 + tt] * 3 + gg) * d.Wt);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&desc_empty[dq]);
            uint32_t t1 = 0, t0 = 0;
            bool ok = true;
            const int chunks = DS.chunks, chunks_case = DS.chunks_case;
            // this group's first stage of the item and its number of stages
            const int kc0 = (int)(((uint64_t)grp + kGroups - (g % kGroups)) % kGroups);
            const int mine = (chunks - kc0 + kGroups - 1) / kGroups;
            // the prefix SNPs' words of this row for the next kPf own stages
            // (a register ring indexed statically: the loop is unrolled by
            // kPf).  Up to order 3 they are kept as loaded and ANDed only
            // when their stage is produced, so no instruction waits for a
            // load issued for a later stage; at orders 4-5 the ring holds the
            // AND (measured: the raw ring's registers spill there, 1586 vs
            // 1527 ms at order 4, 500 x 8192, and 1548 ms with one own stage
            // of prefetch; order 3 combined 94.6 -> 94.0 ms).  EPI_TC_RAW_HI
            // (a prefetch distance) keeps the raw words at every order.
#ifdef EPI_TC_RAW_HI
            constexpr bool kKeepRaw = true;
            constexpr int kPf = km1 <= 2 ? EPI_TC_PREFETCH : EPI_TC_RAW_HI;
#else
            constexpr bool kKeepRaw = km1 <= 2;
            constexpr int kPf = EPI_TC_PREFETCH;
#endif
            constexpr int kRaw = kKeepRaw ? km1 : 1;     // words kept per own stage
            uint4 ring[kPf][kRaw];
            auto fetch = [&](int kc, uint4 *dst) {
                if constexpr (kKeepRaw) {
#pragma unroll
                    for (int tt = 0; tt < km1; tt++) dst[tt] = __ldg(rows[tt] + kc);
                } else {
                    uint4 a = __ldg(rows[0] + kc);
#pragma unroll
                    for (int tt = 1; tt < km1; tt++) {
                        const uint4 v = __ldg(rows[tt] + kc);
                        a.x &= v.x; a.y &= v.y; a.z &= v.z; a.w &= v.w;
                    }
                    dst[0] = a;
                }
            };
#pragma unroll
            for (int u = 0; u < kPf; u++) {
                if (active && u < mine) fetch(kc0 + kGroups * u, ring[u]);
                else {
#pragma unroll
                    for (int tt = 0; tt < kRaw; tt++) ring[u][tt] = make_uint4(0, 0, 0, 0);
                }
            }
            uint64_t gs = g + (uint64_t)kc0;                   // global stage of own stage m
            int s = (int)(gs % kStages);
            uint32_t ph = (uint32_t)((gs / kStages) & 1);
            for (int mb = 0; mb < mine && ok; mb += kPf) {
#pragma unroll
                for (int u = 0; u < kPf; u++) {
                    const int m = mb + u;
                    if (m >= mine) break;
                    const int kc = kc0 + kGroups * m;
                    uint4 cur = ring[u][0];
#pragma unroll
                    for (int tt = 1; tt < kRaw; tt++) {
                        cur.x &= ring[u][tt].x; cur.y &= ring[u][tt].y; cur.z &= ring[u][tt].z; cur.w &= ring[u][tt].w;
                    }
                    if (active && m + kPf < mine) fetch(kc + kGroups * kPf, ring[u]);
                    if (!wait_fast(&empty_ab[s / kRelease], ph ^ 1, &abort_flag, w_prod)) { ok = false; break; }
                    const uint32_t c4 = __popc(cur.x) + __popc(cur.y) + __popc(cur.z) + __popc(cur.w);
                    if (kc < chunks_case) t1 += c4;
                    else t0 += c4;
                    unsigned char *arow = stages_a + s * kTileBytes + r * 128;
                    const uint32_t wv4[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        // output word i = bit i of every byte of the mask word
                        const uint32_t wv = wv4[q];
                        const uint32_t s4 = wv << 4, r4 = wv >> 4;
                        const uint4 lo = make_uint4(s4 & 0x10101010u, s4 & 0x20202020u, s4 & 0x40404040u, wv & 0x08080808u);
                        const uint4 hi = make_uint4(wv & 0x10101010u, wv & 0x20202020u, wv & 0x40404040u, r4 & 0x08080808u);
                        *reinterpret_cast<uint4 *>(arow + (((2 * q) ^ (r & 7)) << 4)) = lo;
                        *reinterpret_cast<uint4 *>(arow + (((2 * q + 1) ^ (r & 7)) << 4)) = hi;
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full_ab[s]);
                    // next own stage: kGroups global stages on
                    s += kGroups;
                    if (s >= kStages) { s -= kStages; ph ^= 1; }
                }
            }
            if (!ok) break;
            g += (uint64_t)chunks;
            const int b = (int)(i & 1);
            const uint32_t ub = (uint32_t)(i >> 1);
            if (!wait_fast(&acc_empty[b], (ub & 1) ^ 1, &abort_flag, w_prod_acc)) break;
            tot[((b * 128 + r) * kMaxProdGroups + grp) * 2 + 0] = t1;
            tot[((b * 128 + r) * kMaxProdGroups + grp) * 2 + 1] = t0;
            __syncwarp();
            if (lane == 0) mbar_arrive(&tot_full[b]);
        }
        if (P.waits && t == 0) {
            P.waits[blockIdx.x * kWaitSlots + 3] = (unsigned long long)w_prod;
            P.waits[blockIdx.x * kWaitSlots + 4] = (unsigned long long)w_prod_acc;
        }
    } else {
        // -------------------------------------------------------- epilogue
        const int quad = warp & 3;           // TMEM lane quadrant
        const int jhalf = warp >> 2;         // column group: chunks jhalf + kCG i of the quadrant
        const int r = quad * 32 + lane;      // tile row = TMEM lane
        const int l = lane;
        const int pos = kWide ? r : l % kPR;          // row of the prefix's table
        const int pl = kWide ? 0 : l / kPR;
        const bool lane_real = kWide ? r < kPR : l < kPPW * kPR;
        const MiConstF32 mc = make_mi_const(d.m, d.m1, d.m0);
        const float vscale = 32.0f * DS.ln2_over_m, voff = DS.tconst * DS.ln2_over_m;
        // combined classes: the decode's control-bit mask and 2^-(p+5)
        const uint32_t lo_mask = (1u << (DS.comb_p & 31)) - 1u;
        const float case_scale = __uint_as_float((uint32_t)(127 - 5 - DS.comb_p) << 23);
        long long w_epi = 0;
        for (int64_t i = 0; i < n_my; i++) {
            const int dq = (int)(i % kDescDepth);
            const uint32_t ud = (uint32_t)(i / kDescDepth);
            const int b = (int)(i & 1);
            const uint32_t ub = (uint32_t)(i >> 1);
            bool ok = mbar_wait(&desc_full[dq], ud & 1, &abort_flag);
            ok = ok && wait_fast(&acc_full[b], ub & 1, &abort_flag, w_epi);
            ok = ok && wait_fast(&tot_full[b], ub & 1, &abort_flag, w_epi);
            ok = __all_sync(0xffffffffu, ok);
            tc_fence_after();
            const Desc &D = desc[dq];
            const int p = quad * kPPW + pl;
            const bool prow = ok && lane_real && p < D.nvalid;
            const int32_t cpre = prow ? D.snp[p * km1 + km1 - 1] : 0x7fffffff;
            int32_t psnp[km1];
#pragma unroll
            for (int tt = 0; tt < km1; tt++) psnp[tt] = prow ? D.snp[p * km1 + tt] : 0;
            // last SNPs of this prefix inside the searched rank range: the
            // combination (prefix, j) has rank base + j.  Only prefixes whose
            // first SNP is the range's first or last can be cut.
            int32_t jlo = cpre + 1, jhi = (int32_t)d.n;
            if (prow && DS.clip && (psnp[0] == DS.s1_lo || psnp[0] == DS.s1_hi)) {
                uint64_t sp = 0;
#pragma unroll
                for (int tt = 0; tt < km1; tt++) sp += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                const int64_t base = (int64_t)DS.total - (int64_t)sp - d.n;
                int64_t lo64 = (int64_t)DS.rank_begin - base, hi64 = (int64_t)DS.rank_end - base;
                lo64 = lo64 < (int64_t)jlo ? (int64_t)jlo : (lo64 > d.n ? d.n : lo64);
                hi64 = hi64 > d.n ? d.n : (hi64 < lo64 ? lo64 : hi64);
                jlo = (int32_t)lo64;
                jhi = (int32_t)hi64;
            }
            // the same interval for the prefixes whose (prefix, last SNP)
            // pairs this lane sums (orders 3-4): pair lane + 32 i is prefix
            // (lane + 32 i) / 8 of the warp and last SNP (lane + 32 i) % 8 of
            // each chunk
            int32_t plo[kPairIters > 0 ? kPairIters : 1], phi[kPairIters > 0 ? kPairIters : 1];
            if constexpr (kTranspose) {
#pragma unroll
                for (int q = 0; q < kPairIters; q++) {
                    const int pp = (lane + 32 * q) >> 3;
                    const int pt = quad * kPPW + pp;
                    plo[q] = 1;
                    phi[q] = 0;                      // empty: no valid last SNP
                    if (ok && pp < kPPW && pt < D.nvalid) {
                        int32_t qs[km1];
#pragma unroll
                        for (int tt = 0; tt < km1; tt++) qs[tt] = D.snp[pt * km1 + tt];
                        plo[q] = qs[km1 - 1] + 1;
                        phi[q] = (int32_t)d.n;
                        if (DS.clip && (qs[0] == DS.s1_lo || qs[0] == DS.s1_hi)) {
                            uint64_t sp = 0;
#pragma unroll
                            for (int tt = 0; tt < km1; tt++) sp += binom_at(d.binom, d.n, d.n - 1 - qs[tt], K - tt);
                            const int64_t base = (int64_t)DS.total - (int64_t)sp - d.n;
                            int64_t lo64 = (int64_t)DS.rank_begin - base, hi64 = (int64_t)DS.rank_end - base;
                            lo64 = lo64 < (int64_t)plo[q] ? (int64_t)plo[q] : (lo64 > d.n ? d.n : lo64);
                            hi64 = hi64 > d.n ? d.n : (hi64 < lo64 ? lo64 : hi64);
                            plo[q] = (int32_t)lo64;
                            phi[q] = (int32_t)hi64;
                        }
                    }
                }
            }
            uint32_t T1 = 0, T0 = 0;
#pragma unroll
            for (int gq = 0; gq < kGroups; gq++) {
                T1 += tot[((b * 128 + r) * kMaxProdGroups + gq) * 2 + 0];
                T0 += tot[((b * 128 + r) * kMaxProdGroups + gq) * 2 + 1];
            }
            // row totals in accumulator units (count / 32, exact)
            const float fT1 = u2f_exact(T1) * 0.03125f, fT0 = u2f_exact(T0) * 0.03125f;
            if (tid == 0) {
                const float gthr = __uint_as_float(*(volatile uint32_t *)DS.global_thr);
                if (ES.list_len == P.pool || gthr > 0.0f) ES.thr = fmaxf(ES.thr, gthr);
            }
            epi_bar<kEpiThreads>();
            float thr = ES.thr, cut = thr - DS.delta;
            int list_len = ES.list_len;
#pragma unroll 1
            for (int jc = 0; jc < kIters; jc++) {
                uint32_t cs[16], cn[16];
                // this warp's chunk of the quadrant: last SNPs j0 .. j0 + 7
                const int jcg = jhalf + kCG * jc;
                const int32_t jb = D.j0 + 8 * jcg;   // the chunk's last SNPs are jb .. jb + 7
                // a chunk past the quadrant's last one, or (orders 3-4) whose
                // first last SNP is past the end (the last N tile of a panel),
                // holds no combination, and its warp skips it (warp-uniform)
                const bool live = ok && jcg < kQC && (!kTranspose || jb < (int32_t)d.n);
                if (live) {
                    // columns 2 (j - D.j0) + g of accumulator b; separate
                    // classes: the control accumulator 128 columns on
                    const uint32_t ta = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 256 + 16 * jcg);
                    if constexpr (C) {
                        uint32_t cc[16];
                        TMEM_LD16(ta, cc);
                        tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 16; q++) split_classes(cc[q], lo_mask, case_scale, cs[q], cn[q]);
                    } else {
                        TMEM_LD16(ta, cs);
                        TMEM_LD16(ta + 128, cn);
                        tmem_wait_ld();
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; q++) { cs[q] = 0; cn[q] = 0; }
                }
                if (jc == kIters - 1) {
                    // every accumulator value is in registers: hand the
                    // buffer back to the MMA issuer before the last scoring
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
                }
                if constexpr (kWide) {
                    // screen sums of the chunk's 8 last SNPs: each warp sums
                    // its rows, the quadrant-0 warp of the half adds the three
                    float vs[8];
#pragma unroll
                    for (int jj = 0; jj < 8; jj++) {
                        const int32_t j = jb + jj;
                        const float fa0 = __uint_as_float(cs[2 * jj]), fa1 = __uint_as_float(cs[2 * jj + 1]);
                        const float fb0 = __uint_as_float(cn[2 * jj]), fb1 = __uint_as_float(cn[2 * jj + 1]);
                        const float fa2 = fT1 - fa0 - fa1, fb2 = fT0 - fb0 - fb1;
                        const bool valid = prow && j >= jlo && j < jhi;
                        if (P.dump && valid) {
                            uint64_t rs = 0;
#pragma unroll
                            for (int tt = 0; tt < km1; tt++) rs += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                            rs += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                            constexpr int cells = kPR * 3;
                            uint32_t *o = P.dump + (DS.total - 1 - rs) * 2 * cells;
                            o[pos * 3 + 0] = f2u_exact(32.0f * fa0); o[pos * 3 + 1] = f2u_exact(32.0f * fa1);
                            o[pos * 3 + 2] = f2u_exact(32.0f * fa2);
                            o[cells + pos * 3 + 0] = f2u_exact(32.0f * fb0);
                            o[cells + pos * 3 + 1] = f2u_exact(32.0f * fb1);
                            o[cells + pos * 3 + 2] = f2u_exact(32.0f * fb2);
                        }
                        float v = 0.0f;
                        if (prow)
                            v = (tlog32(fa0) + tlog32(fb0) - tlog32(fa0 + fb0)) +
                                (tlog32(fa1) + tlog32(fb1) - tlog32(fa1 + fb1)) +
                                (tlog32(fa2) + tlog32(fb2) - tlog32(fa2 + fb2));
                        vs[jj] = warp_sum(v);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) wred[jhalf][quad][jj] = vs[jj];
                    }
                    epi_bar<kEpiThreads>();
                    if (quad == 0 && lane < 8) {
                        const float tv = wred[jhalf][0][lane] + wred[jhalf][1][lane] + wred[jhalf][2][lane] +
                                         wred[jhalf][3][lane];
                        const int32_t j = jb + lane;
                        const bool valid = prow && j >= jlo && j < jhi;
                        wflag[jhalf][lane] = (valid && fmaf(tv, vscale, voff) >= cut) ? 1 : 0;
                    }
                    epi_bar<kEpiThreads>();
                    int anyf = 0;
#pragma unroll
                    for (int q = 0; q < 16; q++) anyf |= wflag[q >> 3][q & 7];
                    if (anyf) {
                        // precise single-precision scores of the flagged sets
#pragma unroll 1
                        for (int jj = 0; jj < 8; jj++) {
                            if (!wflag[jhalf][jj]) continue;
                            float e = 0.0f;
                            if (prow) {
                                const float fa0 = __uint_as_float(cs[2 * jj]), fa1 = __uint_as_float(cs[2 * jj + 1]);
                                const float fb0 = __uint_as_float(cn[2 * jj]), fb1 = __uint_as_float(cn[2 * jj + 1]);
                                e = row_terms_precise(f2u_exact(32.0f * fa0), f2u_exact(32.0f * fb0),
                                                      f2u_exact(32.0f * fa1), f2u_exact(32.0f * fb1),
                                                      f2u_exact(32.0f * (fT1 - fa0 - fa1)),
                                                      f2u_exact(32.0f * (fT0 - fb0 - fb1)), mc);
                            }
                            e = warp_sum(e);
                            if (lane == 0) wpre[jhalf][quad][jj] = e;
                        }
                        epi_bar<kEpiThreads>();
                        if (quad == 0 && lane < 8 && wflag[jhalf][lane]) {
                            const float e = wpre[jhalf][0][lane] + wpre[jhalf][1][lane] + wpre[jhalf][2][lane] +
                                            wpre[jhalf][3][lane];
                            const float score = __fdiv_rn(e, mc.fm);
                            if (score >= thr) {
                                const int32_t j = jb + lane;
                                uint64_t rk_sum = 0;
#pragma unroll
                                for (int tt = 0; tt < km1; tt++)
                                    rk_sum += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                                rk_sum += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                                const int slot = list_len + atomicAdd(&ES.nbuf, 1);
                                sc[slot] = score;
                                rk[slot] = DS.total - 1 - rk_sum;
                            }
                        }
                        epi_bar<kEpiThreads>();
                    }
                } else if constexpr (kTranspose) {
                  if (live) {
                    // row terms of the chunk's 8 last SNPs, straight-line
                    float vrow[8];
#pragma unroll
                    for (int jj = 0; jj < 8; jj++) {
                        // accumulator values x = count / 32 (exact); with
                        // t(x) = x log2 x, T(32 x) = 32 t(x) + 160 x and the
                        // linear parts cancel within a cell, so the screen
                        // sums t over the raw values and scales once
                        const float fa0 = __uint_as_float(cs[2 * jj]), fa1 = __uint_as_float(cs[2 * jj + 1]);
                        const float fb0 = __uint_as_float(cn[2 * jj]), fb1 = __uint_as_float(cn[2 * jj + 1]);
                        const float fa2 = fT1 - fa0 - fa1, fb2 = fT0 - fb0 - fb1;
                        vrow[jj] = prow ? row_screen(fa0, fa1, fa2, fb0, fb1, fb2) : 0.0f;
                    }
                    if (P.dump) {
                        // validation: every table of the chunk, as counts
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) {
                            const int32_t j = jb + jj;
                            if (!(prow && j >= jlo && j < jhi)) continue;
                            const float fa0 = __uint_as_float(cs[2 * jj]), fa1 = __uint_as_float(cs[2 * jj + 1]);
                            const float fb0 = __uint_as_float(cn[2 * jj]), fb1 = __uint_as_float(cn[2 * jj + 1]);
                            uint64_t rs = 0;
#pragma unroll
                            for (int tt = 0; tt < km1; tt++) rs += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                            rs += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                            constexpr int cells = kPR * 3;
                            uint32_t *o = P.dump + (DS.total - 1 - rs) * 2 * cells;
                            o[pos * 3 + 0] = f2u_exact(32.0f * fa0); o[pos * 3 + 1] = f2u_exact(32.0f * fa1);
                            o[pos * 3 + 2] = f2u_exact(32.0f * (fT1 - fa0 - fa1));
                            o[cells + pos * 3 + 0] = f2u_exact(32.0f * fb0);
                            o[cells + pos * 3 + 1] = f2u_exact(32.0f * fb1);
                            o[cells + pos * 3 + 2] = f2u_exact(32.0f * (fT0 - fb0 - fb1));
                        }
                    }
                    // transpose: lane l's 8 values at [l][0..7]; the lane of
                    // pair (prefix pp, last SNP jj) reads rows pp*kPR .. of
                    // column jj (banks 8 (pp kPR + r) + jj: distinct over the
                    // warp's pairs)
                    float *wb = wsum + warp * 256;
                    reinterpret_cast<float4 *>(wb + lane * 8)[0] = make_float4(vrow[0], vrow[1], vrow[2], vrow[3]);
                    reinterpret_cast<float4 *>(wb + lane * 8)[1] = make_float4(vrow[4], vrow[5], vrow[6], vrow[7]);
                    __syncwarp();
                    uint32_t cmask[kPairIters];
#pragma unroll
                    for (int q = 0; q < kPairIters; q++) {
                        const int pair = lane + 32 * q;
                        bool cand = false;
                        if (pair < kPairs) {
                            const int pp = pair >> 3, jj = pair & 7;
                            float v = 0.0f, w2 = 0.0f;
#pragma unroll
                            for (int rr = 0; rr < kPR; rr++) {
                                if (rr & 1) w2 += wb[(pp * kPR + rr) * 8 + jj];
                                else v += wb[(pp * kPR + rr) * 8 + jj];
                            }
                            v += w2;
                            const int32_t j = jb + jj;
                            cand = j >= plo[q] && j < phi[q] && fmaf(v, vscale, voff) >= cut;
                        }
                        cmask[q] = __ballot_sync(0xffffffffu, cand);
                    }
                    __syncwarp();
                    // precise single-precision scores of the flagged pairs
                    // (rare): the prefix's row lanes score their rows of that
                    // column, the prefix's first row lane adds them up
#pragma unroll
                    for (int q = 0; q < kPairIters; q++) {
                        while (cmask[q]) {
                            const int pair = __ffs(cmask[q]) - 1 + 32 * q;
                            cmask[q] &= cmask[q] - 1;
                            const int pp = pair >> 3, jsel = pair & 7;
                            uint32_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
#pragma unroll
                            for (int jj = 0; jj < 8; jj++)
                                if (jj == jsel) { a0 = cs[2 * jj]; a1 = cs[2 * jj + 1]; b0 = cn[2 * jj]; b1 = cn[2 * jj + 1]; }
                            const float fa0 = __uint_as_float(a0), fa1 = __uint_as_float(a1);
                            const float fb0 = __uint_as_float(b0), fb1 = __uint_as_float(b1);
                            float e = 0.0f;
                            if (lane_real && pl == pp)
                                e = row_terms_precise(f2u_exact(32.0f * fa0), f2u_exact(32.0f * fb0),
                                                      f2u_exact(32.0f * fa1), f2u_exact(32.0f * fb1),
                                                      f2u_exact(32.0f * (fT1 - fa0 - fa1)),
                                                      f2u_exact(32.0f * (fT0 - fb0 - fb1)), mc);
                            e = seg_sum<kPR>(e, pos);
                            if (lane_real && pl == pp && pos == 0) {
                                const float score = __fdiv_rn(e, mc.fm);
                                if (score >= thr) {
                                    const int32_t j = jb + jsel;
                                    uint64_t rk_sum = 0;
#pragma unroll
                                    for (int tt = 0; tt < km1; tt++)
                                        rk_sum += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                                    rk_sum += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                                    const int slot = list_len + atomicAdd(&ES.nbuf, 1);
                                    sc[slot] = score;
                                    rk[slot] = DS.total - 1 - rk_sum;
                                }
                            }
                        }
                    }
                  }
                } else {
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const int32_t j = jb + jj;
                    // accumulator values x = count / 32 (exact); with
                    // t(x) = x log2 x, T(32 x) = 32 t(x) + 160 x and the
                    // linear parts cancel within a cell, so the screen sums
                    // t over the raw values and scales once
                    const float fa0 = __uint_as_float(cs[2 * jj]), fa1 = __uint_as_float(cs[2 * jj + 1]);
                    const float fb0 = __uint_as_float(cn[2 * jj]), fb1 = __uint_as_float(cn[2 * jj + 1]);
                    const float fa2 = fT1 - fa0 - fa1, fb2 = fT0 - fb0 - fb1;
                    const bool valid = prow && j >= jlo && j < jhi;
                    if (P.dump && valid) {
                        const uint32_t a0 = f2u_exact(32.0f * fa0), a1 = f2u_exact(32.0f * fa1),
                                       a2 = f2u_exact(32.0f * fa2);
                        const uint32_t b0 = f2u_exact(32.0f * fb0), b1 = f2u_exact(32.0f * fb1),
                                       b2 = f2u_exact(32.0f * fb2);
                        uint64_t rs = 0;
#pragma unroll
                        for (int tt = 0; tt < km1; tt++) rs += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                        rs += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                        constexpr int cells = kPR * 3;
                        uint32_t *o = P.dump + (DS.total - 1 - rs) * 2 * cells;
                        o[pos * 3 + 0] = a0; o[pos * 3 + 1] = a1; o[pos * 3 + 2] = a2;
                        o[cells + pos * 3 + 0] = b0; o[cells + pos * 3 + 1] = b1; o[cells + pos * 3 + 2] = b2;
                    }
                    float v = 0.0f;
                    if (prow)
                        v = (tlog32(fa0) + tlog32(fb0) - tlog32(fa0 + fb0)) +
                            (tlog32(fa1) + tlog32(fb1) - tlog32(fa1 + fb1)) +
                            (tlog32(fa2) + tlog32(fb2) - tlog32(fa2 + fb2));
                    v = seg_sum<kPR>(v, pos);
                    const float approx = fmaf(v, vscale, voff);
                    const bool cand = valid && pos == 0 && approx >= cut;
                    uint32_t seg_mask = __ballot_sync(0xffffffffu, cand);
                    while (seg_mask) {
                        const int leader = __ffs(seg_mask) - 1;
                        seg_mask &= seg_mask - 1;
                        float e = 0.0f;
                        if (l / kPR == leader / kPR && lane_real)
                            e = row_terms_precise(f2u_exact(32.0f * fa0), f2u_exact(32.0f * fb0),
                                                  f2u_exact(32.0f * fa1), f2u_exact(32.0f * fb1),
                                                  f2u_exact(32.0f * fa2), f2u_exact(32.0f * fb2), mc);
                        e = seg_sum<kPR>(e, pos);
                        if (l == leader) {
                            const float score = __fdiv_rn(e, mc.fm);
                            if (score >= thr) {
                                uint64_t rk_sum = 0;
#pragma unroll
                                for (int tt = 0; tt < km1; tt++)
                                    rk_sum += binom_at(d.binom, d.n, d.n - 1 - psnp[tt], K - tt);
                                rk_sum += binom_at(d.binom, d.n, d.n - 1 - j, 1);
                                const int slot = list_len + atomicAdd(&ES.nbuf, 1);
                                sc[slot] = score;
                                rk[slot] = DS.total - 1 - rk_sum;
                            }
                        }
                    }
                }
                }
                if (jc % kJcPerCheck == kJcPerCheck - 1) {
                    epi_bar<kEpiThreads>();
                    // the next check interval adds at most kJcPerCheck chunks
                    // of 8 last SNPs per column group and prefix of the tile:
                    // sort and trim first if the buffer could not hold them
                    if (ES.list_len + ES.nbuf + kJcPerCheck * 8 * kCG * kPPT > P.cand_p2)
                        epi_flush<kEpiThreads>(ES, sc, rk, P.pool, DS.global_thr, tid);
                    thr = ES.thr;
                    cut = thr - DS.delta;
                    list_len = ES.list_len;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&desc_empty[dq]);
            epi_bar<kEpiThreads>();
            if (tid == 0) ES.stop = abort_flag;
            epi_bar<kEpiThreads>();
            if (ES.stop) break;
        }
        epi_bar<kEpiThreads>();
        if (ES.nbuf > 0) epi_flush<kEpiThreads>(ES, sc, rk, P.pool, DS.global_thr, tid);
        const int L = ES.list_len;
        for (int q = tid; q < L; q += kEpiThreads) {
            P.list_score[(size_t)blockIdx.x * P.pool + q] = sc[q];
            P.list_rank[(size_t)blockIdx.x * P.pool + q] = rk[q];
        }
        if (tid == 0) P.list_count[blockIdx.x] = L;
        if (P.waits && tid == 0) P.waits[blockIdx.x * kWaitSlots + 5] = (unsigned long long)w_epi;
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kWarpMma) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
    if (tid == 0 && abort_flag) atomicOr(P.status, ST_TIMEOUT);
}

// Prefixes searched per panel (first SNP in [a, b]) and their exclusive
// prefix sum over c into pcum; then items per panel (the M tiles whose first
// prefix lies in panel c, times the N tiles of that panel) and their
// exclusive prefix sum into cum.  One block.
__device__ __forceinline__ uint64_t panel_prefixes(const DevData &d, int k, int64_t c, int64_t a, int64_t b)
{
    if (c < k - 2 || c > d.n - 2) return 0;
    if (k == 2) return (c >= a && c <= b) ? 1 : 0;
    return subsets_from(d, c, a, k - 2) - subsets_from(d, c, b + 1, k - 2);
}

__device__ void block_exclusive_scan(uint64_t *part, uint64_t s, uint64_t &before, uint64_t &total)
{
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    before = part[threadIdx.x] - s;
    total = part[1023];
    __syncthreads();
}

__global__ void __launch_bounds__(1024) item_cum_kernel(DevData d, int k, int ppt, int kj, int32_t a, int32_t b,
                                                        uint64_t *pcum, uint64_t *cum)
{
    __shared__ uint64_t part[1024];
    const int64_t n = d.n;
    const int64_t per = (n + 1023) / 1024;
    const int64_t cb = (int64_t)threadIdx.x * per, ce = min(n, cb + per);
    uint64_t s = 0, run = 0, all = 0;
    for (int64_t c = cb; c < ce; c++) s += panel_prefixes(d, k, c, a, b);
    block_exclusive_scan(part, s, run, all);
    for (int64_t c = cb; c < ce; c++) {
        pcum[c] = run;
        run += panel_prefixes(d, k, c, a, b);
    }
    if (threadIdx.x == 1023) pcum[n] = all;
    __syncthreads();
    auto items = [&](int64_t c) -> uint64_t {
        if (c < k - 2 || c > n - 2) return 0;
        const uint64_t t0 = (pcum[c] + ppt - 1) / ppt;
        const uint64_t t1 = (pcum[c + 1] + ppt - 1) / ppt;
        return (t1 - t0) * (uint64_t)((n - 1 - c + kj - 1) / kj);
    };
    s = 0;
    for (int64_t c = cb; c < ce; c++) s += items(c);
    block_exclusive_scan(part, s, run, all);
    for (int64_t c = cb; c < ce; c++) {
        cum[c] = run;
        run += items(c);
    }
    if (threadIdx.x == 1023) cum[n] = all;
}

// B operand: row 2j+g (g = 0, 1) of SNP j, K byte 32 w + 4 i + b = individual
// 32 w + 8 b + i (the A producer's order); where the genotype is g the byte
// is a power of two, else 0.  The producer's A bytes by position i are 0x10,
// 0x20, 0x40, 0x08 (twice), and B's are 0x38, 0x28, 0x08, 0x40:
//   read as E4M3, A = 2^-5, 2^-3, 2^1, 2^-6 and B = 2^0, 2^-2, 2^-6, 2^1, so
//   every product of two ones is 2^-5 (separate-class variant, case_shift 0);
//   read as E5M2, A = 2^-11, 2^-7, 2^1, 2^-13 and B = 2^-1, 2^-5, 2^-13,
//   2^1, so every product is 2^-12; the case words (w < W1) add p to B's
//   exponent field (case_shift = 4 p, p <= 14 keeps it finite), making their
//   products 2^(p-12) (combined-class variant).
__global__ void build_b8_kernel(DevData d, unsigned char *__restrict__ b8, uint32_t case_shift)
{
    const uint32_t bval[8] = {0x38u, 0x28u, 0x08u, 0x40u, 0x38u, 0x28u, 0x08u, 0x40u};
    const int64_t Kt = (int64_t)d.Wt * 32;
    const int64_t per_row = Kt / 16;
    const int64_t total = 2 * d.n * per_row;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = idx / per_row;
        const int64_t q = idx - row * per_row;            // 16-byte piece
        const int64_t j = row >> 1;
        const int g = (int)(row & 1);
        const uint32_t word = d.masks[(j * 3 + g) * d.Wt + (q >> 1)];
        const int i0 = (int)(q & 1) * 4;
        const uint32_t add = (q >> 1) < d.W1 ? case_shift : 0u;
        uint32_t o[4];
#pragma unroll
        for (int t = 0; t < 4; t++) o[t] = ((word >> (i0 + t)) & 0x01010101u) * (bval[i0 + t] + add);
        reinterpret_cast<uint4 *>(b8)[idx] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

}  // namespace tc

// ----------------------------------------------------------------- host --
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encode()
{
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

size_t tc_b8_bytes(const DevData &d) { return (size_t)2 * d.n * d.Wt * 32; }

cudaError_t launch_build_b8(const DevData &d, unsigned char *b8, int num_sms, cudaStream_t st, int comb_p)
{
    const int64_t total = 2 * d.n * (int64_t)d.Wt * 2;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    tc::build_b8_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(d, b8, 4u * (uint32_t)comb_p);
    return cudaGetLastError();
}

// Class shift p of the combined-class variant for an order-k search of d, or
// 0 where it does not apply: order 3 (at order 4 its single producer group
// bounds it, measured slower than separate classes); the control count must
// fit below 2^p and the accumulator value ctrl + case 2^p below 2^23 (the
// decode's exact range; FP32 accumulation of such integers is exact).
int tc_comb_shift(const DevData &d, int k)
{
    if (k != 3) return 0;
    int p = 1;
    while (p < 15 && (1ll << p) <= d.m0) p++;
    if (p > 14) return 0;
    if (d.m1 * (1ll << p) + d.m0 >= (1ll << 23)) return 0;
    return p;
}

static int tc_pr(int k) { return k == 2 ? 3 : (k == 3 ? 9 : (k == 4 ? 27 : 81)); }
static int tc_ppt(int k) { return tc_pr(k) > 32 ? 1 : 4 * (32 / tc_pr(k)); }

// Work items of an order-k search over first SNPs [a, b] (same formulas as
// item_cum_kernel): the host needs the count to split items over the CTAs.
static uint64_t host_subsets_from(int64_t c, int64_t x, int m)
{
    if (m == 0) return 1;
    return c - x >= m ? host_binom(c - x, m) : 0;
}

uint64_t tc_item_count(int64_t n, int k, int64_t a, int64_t b, int kj)
{
    const uint64_t ppt = (uint64_t)tc_ppt(k);
    uint64_t total = 0, pc = 0;
    for (int64_t c = k - 2; c <= n - 2; c++) {
        uint64_t cnt;
        if (k == 2) cnt = (c >= a && c <= b) ? 1 : 0;
        else cnt = host_subsets_from(c, a, k - 2) - host_subsets_from(c, b + 1, k - 2);
        const uint64_t t0 = (pc + ppt - 1) / ppt;
        pc += cnt;
        const uint64_t t1 = (pc + ppt - 1) / ppt;
        total += (t1 - t0) * (uint64_t)((n - 1 - c + kj - 1) / kj);
    }
    return total;
}

uint64_t tc_item_count(int64_t n, int k) { return tc_item_count(n, k, 0, n - k, tc::Shape<false>::J); }

// First SNP of the combination of lexicographic rank r: the largest s with
// C(n, k) - C(n - s, k) <= r (the combinations starting below s come first).
int64_t tc_first_snp(int64_t n, int k, uint64_t r)
{
    const uint64_t total = host_binom(n, k);
    int64_t lo = 0, hi = n - k;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (total - host_binom(n - mid, k) <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Combinations the tensor path counts for the rank range [rb, re): every
// combination whose first SNP lies in [first SNP of rb, first SNP of re - 1].
uint64_t tc_range_work(int64_t n, int k, uint64_t rb, uint64_t re)
{
    if (re <= rb) return 0;
    const int64_t a = tc_first_snp(n, k, rb), b = tc_first_snp(n, k, re - 1);
    // combinations whose first SNP is >= a, minus those whose first SNP is > b
    return host_binom(n - a, k) - host_binom(n - b - 1, k);
}

int tc_prefixes_per_warp(int k)
{
    const int PR = k == 2 ? 3 : (k == 3 ? 9 : (k == 4 ? 27 : 81));
    return PR <= 32 ? 32 / PR : 0;
}

// Candidate buffer entries: the pool plus one check interval (2 chunks of 8
// last SNPs, both halves, every prefix of the tile; order 2 checks every
// chunk), rounded up to a power of two for the bitonic sort.
int tc_cand_p2(int k, int pool, bool comb)
{
    const int groups = tc::roles_epi_warps(comb, k) / 4;
    const int check = k == 2 ? 1 : tc::roles_check_iters(comb, k);
    return next_pow2(pool + check * 8 * groups * tc_ppt(k));
}

size_t tc_smem_bytes(int cand_p2, int k, bool cand_global, bool comb)
{
    const size_t transpose =
        (k == 3 || k == 4) ? (size_t)tc::roles_epi_warps(comb, k) * 256 * 4 + 16 : 0;
    const size_t rings = comb ? (size_t)tc::Shape<true>::Stages * (tc::kTileBytes + tc::Shape<true>::BBytes)
                              : (size_t)tc::Shape<false>::Stages * (tc::kTileBytes + tc::Shape<false>::BBytes);
    return 1024 + rings + (cand_global ? 0 : (size_t)cand_p2 * 12) + 2 * 128 * tc::kMaxProdGroups * 2 * 4 +
           tc::kDescDepth * sizeof(tc::Desc) + 64 + transpose;
}


static cudaError_t encode_map(CUtensorMap *map, const DevData &d, const unsigned char *b8, bool comb)
{
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    const int64_t Kt = (int64_t)d.Wt * 32;
    cuuint64_t gdim[2] = {(cuuint64_t)Kt, (cuuint64_t)(2 * d.n)};
    cuuint64_t gstride[1] = {(cuuint64_t)Kt};
    cuuint32_t box[2] = {(cuuint32_t)tc::kKC, comb ? (cuuint32_t)tc::Shape<true>::N : (cuuint32_t)tc::Shape<false>::N};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult cr = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<unsigned char *>(b8), gdim, gstride, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Per-dataset parameters (host side); the B-operand map goes to tmap_dev when
// the launch is batched (nullptr: passed as a kernel parameter instead).
static void fill_ds(tc::DsParams &D, const DevData &d, int k, uint64_t *item_cum, uint32_t *global_thr,
                    uint64_t total, uint64_t rb, uint64_t re, const CUtensorMap *tmap_dev, int cta_begin,
                    int cta_count, int comb_p)
{
    D.d = d;
    D.comb_p = comb_p;
    D.rank_begin = rb;
    D.rank_end = re;
    D.s1_lo = (int32_t)tc_first_snp(d.n, k, rb);
    D.s1_hi = (int32_t)tc_first_snp(d.n, k, re - 1);
    D.clip = !(rb == 0 && re == total);
    // prefixes whose first SNP lies in [s1_lo, s1_hi]
    uint64_t np = 0;
    for (int64_t c = k - 2; c <= d.n - 2; c++) {
        if (k == 2) np += (c >= D.s1_lo && c <= D.s1_hi) ? 1 : 0;
        else np += host_subsets_from(c, D.s1_lo, k - 2) - host_subsets_from(c, D.s1_hi + 1, k - 2);
    }
    D.n_prefix = np;
    D.n_items = tc_item_count(d.n, k, D.s1_lo, D.s1_hi, comb_p ? tc::Shape<true>::J : tc::Shape<false>::J);
    D.item_cum = item_cum;
    D.pcum = item_cum + d.n + 1;
    const int64_t Kt = (int64_t)d.Wt * 32;
    D.chunks = (int)(Kt / tc::kKC);
    D.chunks_case = (int)((int64_t)d.W1 * 32 / tc::kKC);
    auto T = [](double c) { return c > 0 ? c * log2(c) : 0.0; };
    D.tconst = (float)(T((double)d.m) - T((double)d.m1) - T((double)d.m0));
    D.ln2_over_m = (float)(0.6931471805599453 / (double)d.m);
    // screening margin: relative errors of the log2 approximation (2^-21)
    // and of the float sums over (T(m) + T(m1) + T(m0)), doubled
    const int64_t cells = (int64_t)tc_pr(k) * 3;
    // bound on the summed magnitudes of the screen's terms: with t(x) =
    // T(32 x) / 32 - 5 x over accumulator values x = count / 32, 32 sum |t|
    // <= sum T(c) + 5 sum c <= T(m) + T(m1) + T(m0) + 10 m
    const double mag = T((double)d.m) + T((double)d.m1) + T((double)d.m0) + 10.0 * (double)d.m;
    D.delta = (float)(2.0 * (4.0 * 4.76837158203125e-7 + (double)(2 * cells + 40) * 5.9604644775390625e-8) * mag *
                      0.6931471805599453 / (double)d.m) + 1e-7f;
    D.total = total;
    D.global_thr = global_thr;
    D.tmap = tmap_dev;
    D.cta_begin = cta_begin;
    D.cta_count = cta_count;
}

static void fill_launch(tc::Params &P, int k, int pool, float *list_score, uint64_t *list_rank, int32_t *list_count,
                        int32_t *status, uint32_t *dump, unsigned long long *waits, float *cand_g,
                        uint64_t *rank_g, bool comb)
{
    P.k = k;
    P.PR = tc_pr(k);
    P.ppw = P.PR > 32 ? 0 : 32 / P.PR;
    P.ppt = tc_ppt(k);
    P.pool = pool;
    P.cand_p2 = tc_cand_p2(k, pool, comb);
    P.cand_score_g = cand_g;
    P.cand_rank_g = rank_g;
    P.wait_ns = 0;
    P.list_score = list_score;
    P.list_rank = list_rank;
    P.list_count = list_count;
    P.status = status;
    P.dump = dump;
    P.waits = waits;
}

static cudaError_t launch_kernel(const CUtensorMap &map, const tc::Params &P, int k, int grid, cudaStream_t st,
                                 bool comb)
{
    const size_t smem = tc_smem_bytes(P.cand_p2, k, P.cand_score_g != nullptr, comb);
    auto kern = k == 2   ? tc::tc_search_kernel<2, false>
                : k == 3 ? (comb ? tc::tc_search_kernel<3, true> : tc::tc_search_kernel<3, false>)
                : k == 4 ? tc::tc_search_kernel<4, false>
                         : tc::tc_search_kernel<5, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = comb ? tc::Roles<true, 3>::Threads
                             : (k == 4 ? tc::Roles<false, 4>::Threads : tc::Roles<false, 3>::Threads);
    kern<<<grid, threads, smem, st>>>(map, P);
    return cudaGetLastError();
}

cudaError_t launch_tc_item_cum(const DevData &d, int k, uint64_t rb, uint64_t re, uint64_t *item_cum,
                               cudaStream_t st, bool comb)
{
    const int32_t a = (int32_t)tc_first_snp(d.n, k, rb), b = (int32_t)tc_first_snp(d.n, k, re - 1);
    const int kj = comb ? tc::Shape<true>::J : tc::Shape<false>::J;
    tc::item_cum_kernel<<<1, 1024, 0, st>>>(d, k, tc_ppt(k), kj, a, b, item_cum + d.n + 1, item_cum);
    return cudaGetLastError();
}

cudaError_t launch_tc_search(const DevData &d, int k, const unsigned char *b8, uint64_t *item_cum, int pool,
                             uint32_t *global_thr, float *list_score, uint64_t *list_rank, int32_t *list_count,
                             int32_t *status, int grid, uint64_t total, uint64_t rb, uint64_t re, cudaStream_t st,
                             int *cand_p2_out, float *cand_g, uint64_t *rank_g, uint32_t *dump,
                             unsigned long long *waits, unsigned long long wait_ns, int comb_p)
{
    tc::Params P;
    fill_ds(P.one, d, k, item_cum, global_thr, total, rb, re, nullptr, 0, grid, comb_p);
    P.many = nullptr;
    P.cta_ds = nullptr;
    fill_launch(P, k, pool, list_score, list_rank, list_count, status, dump, waits, cand_g, rank_g, comb_p != 0);
    P.wait_ns = wait_ns;
    *cand_p2_out = P.cand_p2;
    cudaError_t e = launch_tc_item_cum(d, k, rb, re, item_cum, st, comb_p != 0);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    e = encode_map(&map, d, b8, comb_p != 0);
    if (e != cudaSuccess) return e;
    return launch_kernel(map, P, k, grid, st, comb_p != 0);
}

size_t tc_ds_bytes() { return sizeof(tc::DsParams); }

cudaError_t tc_fill_batch_entry(void *ds_host, void *tmap_host, const DevData &d, int k, const unsigned char *b8,
                                uint64_t *item_cum, uint32_t *global_thr, uint64_t total, const void *tmap_dev,
                                int cta_begin, int cta_count)
{
    fill_ds(*static_cast<tc::DsParams *>(ds_host), d, k, item_cum, global_thr, total, 0, total,
            static_cast<const CUtensorMap *>(tmap_dev), cta_begin, cta_count, 0);
    return encode_map(static_cast<CUtensorMap *>(tmap_host), d, b8, false);
}

cudaError_t launch_tc_batch(const void *ds_dev, const int32_t *cta_ds_dev, int k, int pool, float *list_score,
                            uint64_t *list_rank, int32_t *list_count, int32_t *status, int grid, cudaStream_t st,
                            float *cand_g, uint64_t *rank_g)
{
    tc::Params P;
    P.one = tc::DsParams();
    P.many = static_cast<const tc::DsParams *>(ds_dev);
    P.cta_ds = cta_ds_dev;
    fill_launch(P, k, pool, list_score, list_rank, list_count, status, nullptr, nullptr, cand_g, rank_g, false);
    CUtensorMap unused;
    memset(&unused, 0, sizeof(unused));
    return launch_kernel(unused, P, k, grid, st, false);
}

}  // namespace epi
