// Internal declarations of libepi shared by its CUDA translation units.
//
// Device data layout of a dataset (the genotype tables of Section 2.1):
//   masks  uint32 [n][3][Wt]  row g of SNP s: bit b of word w is individual
//                             32 w + b; words [0, W1) hold the cases,
//                             [W1, Wt) the controls (each subtable in input
//                             order, zero padded to a multiple of 128 bits)
//   binom  uint64 [9][n + 1]  C(a, b) for 0 <= a <= n, 0 <= b <= 8
// A combination's flat index is its lexicographic rank; consecutive ranks
// share their (k-1)-prefix and differ in the last SNP, as in the
// depth-first order of Algorithm 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/epi.h"

namespace epi {

constexpr int kMaxOrderGpu = 8;          // orders of the popcount search kernels
constexpr int kMaxOrderTc = 5;           // orders of the tensor-core search
constexpr int kMaxPoolLists = 8192;      // entries of one candidate list
constexpr uint64_t kBinomSaturated = ~0ull;

// device status bits (OR-ed by kernels, read by the host after a call)
enum : int32_t {
    ST_BAD_GENO = 1,
    ST_BAD_PHENO = 2,
    ST_POOL_OVERFLOW = 4,
    ST_TIMEOUT = 8,
    ST_INTERNAL = 16,
};

struct DevData {
    int64_t n, m, m1, m0;
    int32_t W1, W0, Wt;          // uint32 words per subtable row
    const uint32_t *masks;       // [n][3][Wt]
    const uint64_t *binom;       // [9][n+1]
};

__host__ __device__ inline uint64_t binom_at(const uint64_t *tab, int64_t n, int64_t a, int b)
{
    if (b < 0 || a < b || a < 0) return 0;
    return tab[(int64_t)b * (n + 1) + a];
}

// Lexicographic unranking of r among the k-subsets of [0, n) (count of
// subsets whose element t is below c is C(n-start, k-t) - C(n-c, k-t)).
__device__ inline void unrank_lex(const uint64_t *tab, int64_t n, int k, uint64_t r, int32_t *out)
{
    int64_t start = 0;
    for (int t = 0; t < k; t++) {
        const int rem = k - t;                       // elements still to place
        const uint64_t total = binom_at(tab, n, n - start, rem);
        const uint64_t x = total - r;                // >= 1
        // smallest c in [start, n-rem] with C(n-1-c, rem) < x
        int64_t lo = start, hi = n - rem;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (binom_at(tab, n, n - 1 - mid, rem) < x) hi = mid;
            else lo = mid + 1;
        }
        r -= total - binom_at(tab, n, n - lo, rem);
        out[t] = (int32_t)lo;
        start = lo + 1;
    }
}

// ---------------------------------------------------------------------------
// Mutual information per cell.
//
// Eq. 1 written as a sum of non-negative terms: with e = n_x m_y / m the
// count expected under independence and u = n / e - 1,
//     m * MI = sum over cells and classes of  e * phi(u),
//     phi(u) = (1 + u) ln(1 + u) - u  >= 0,
// because n ln(n/e) = e phi(u) + (n - e) and the (n - e) sum to zero within
// each cell.  Every term is >= 0, so the sum has no cancellation and the
// single-precision value keeps a small relative error even when MI is small.
// phi is evaluated through y = u / (2 + u), ln(1+u) = 2 atanh(y):
//     phi(u) = u y + 2 (1 + u) y (y^2/3 + y^4/5 + ...)
// for |y| <= 1/2, and directly as (1+u) log1p(u) - u elsewhere (no
// cancellation there).  log1p is CUDA's.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float phi_f32(float u)
{
    if (u >= -0.6666667f && u <= 2.0f) {
        const float y = u * __frcp_rn(2.0f + u);
        const float y2 = y * y;
        float s = 1.0f / 23.0f;
        s = fmaf(s, y2, 1.0f / 21.0f);
        s = fmaf(s, y2, 1.0f / 19.0f);
        s = fmaf(s, y2, 1.0f / 17.0f);
        s = fmaf(s, y2, 1.0f / 15.0f);
        s = fmaf(s, y2, 1.0f / 13.0f);
        s = fmaf(s, y2, 1.0f / 11.0f);
        s = fmaf(s, y2, 1.0f / 9.0f);
        s = fmaf(s, y2, 1.0f / 7.0f);
        s = fmaf(s, y2, 1.0f / 5.0f);
        s = fmaf(s, y2, 1.0f / 3.0f);
        s *= y2;
        return fmaf(2.0f * (1.0f + u) * y, s, u * y);
    }
    return fmaf(1.0f + u, log1pf(u), -u);
}

__device__ __forceinline__ double phi_f64(double u)
{
    if (u >= -0.25 && u <= 0.4) {
        // |y| <= 1/6.9: 14 terms reach double precision
        const double y = u / (2.0 + u);
        const double y2 = y * y;
        double s = 1.0 / 29.0;
        for (int d = 27; d >= 3; d -= 2) s = fma(s, y2, 1.0 / d);
        s *= y2;
        return fma(2.0 * (1.0 + u) * y, s, u * y);
    }
    return fma(1.0 + u, log1p(u), -u);
}

// Approximate log2 of a normal float (the PTX instruction, flushing
// subnormal inputs: the callers' arguments are at least 1/32, so the flush
// never applies and no subnormal handling is emitted around it).  Error:
// at most 2^-22 absolute for x in [0.5, 2], 2 ulp of the result elsewhere.
__device__ __forceinline__ float lg2n(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact float of an integer below 2^23 without a conversion instruction:
// 2^23 + v has v as its mantissa.
__device__ __forceinline__ float u2f_exact(uint32_t v)
{
    return __int_as_float(0x4B000000u | v) - 8388608.0f;
}

// Constants of one dataset for the single-precision cell terms.
struct MiConstF32 {
    float fm, fm1, fm0;       // class sizes as exact floats (< 2^23)
    float inv_m, inv_m1, inv_m0;
};

__device__ __forceinline__ MiConstF32 make_mi_const(int64_t m, int64_t m1, int64_t m0)
{
    MiConstF32 c;
    c.fm = (float)m; c.fm1 = (float)m1; c.fm0 = (float)m0;
    c.inv_m = 1.0f / c.fm;
    c.inv_m1 = m1 ? 1.0f / c.fm1 : 0.0f;
    c.inv_m0 = m0 ? 1.0f / c.fm0 : 0.0f;
    return c;
}

// e * phi(u) of one class in a cell: n = count, fx = cell total (float),
// rx = 1 / fx, fmy / inv_my = class size and its inverse.  With p = fx * fmy
// and err its exact rounding error (fma), m (n - e) = n m - nx my is
// fma(n, m, -p) - err to about one ulp however strong the cancellation.
__device__ __forceinline__ float class_term_f32(uint32_t n, float fx, float rx, float fmy, float inv_my,
                                                const MiConstF32 &c)
{
    if (fmy == 0.0f) return 0.0f;
    const float p = fx * fmy;
    const float err = fmaf(fx, fmy, -p);
    const float e = p * c.inv_m;
    if (n == 0) return e;                           // phi(-1) = 1
    const float num = fmaf(u2f_exact(n), c.fm, -p) - err;
    const float u = num * rx * inv_my;
    return e * phi_f32(u);
}

// Both classes of one cell (a cases, b controls).
__device__ __forceinline__ float cell_terms_f32(uint32_t a, uint32_t b, const MiConstF32 &c)
{
    const uint32_t nx = a + b;
    if (nx == 0) return 0.0f;
    const float fx = u2f_exact(nx);
    const float rx = __frcp_rn(fx);
    return class_term_f32(a, fx, rx, c.fm1, c.inv_m1, c) + class_term_f32(b, fx, rx, c.fm0, c.inv_m0, c);
}

// Compensated running sum of non-negative terms (Neumaier's variant of
// Kahan summation): the exact rounding error of each addition (Fast2Sum,
// larger operand first) is carried in c, so a long sum of cell terms keeps
// the per-term accuracy instead of growing with the number of cells.
struct SumF32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float big = fmaxf(s, x), small = fminf(s, x);
        const float t = big + small;
        c += small - (t - big);
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

__device__ __forceinline__ double mi_term_f64(uint32_t n, uint32_t nx, int64_t my, int64_t m)
{
    if (nx == 0 || my == 0) return 0.0;
    const int64_t den = (int64_t)nx * my;
    const double e = (double)den / (double)m;
    if (n == 0) return e;
    const int64_t num = (int64_t)n * m - den;
    return e * phi_f64((double)num / (double)den);
}

// Relative bound on |MI_f32 - MI| / MI of the single-precision score of an
// order-k table over m individuals (u = 2^-24), the margin of the exact
// top-N proof.  Per term e phi(v) of the sum:
//   * e = (n_x m_y) / m: 3 roundings;
//   * v = n / e - 1: 6 roundings (numerator formed as fma(n, m, -p) - err
//     and its two roundings, the reciprocals 1 / n_x and 1 / m_y, two
//     products), amplified by the condition number v phi'(v) / phi(v) =
//     v ln(1+v) / phi(v), which is 2 near v = 0, tends to 1 for large v and
//     grows like ln(e / n) <= ln m as v -> -1 (n >= 1; n = 0 is exact);
//   * phi(v): at most 9 roundings' worth (series branch: the reciprocal,
//     Horner steps whose terms shrink by y^2 <= 1/4, the final fma; log1p
//     branch: log1pf's ulp and two roundings times the cancellation
//     (1+v) ln(1+v) / phi(v) <= 2.6 at v >= 2);
//   * the product e phi: 1.
// So one term carries at most (3 + 6 (2 + ln m) + 9 + 1) u = (25 + 6 ln m) u.
// The L = 2 3^k non-negative terms are summed either compensated (error
// 2u + 2 L^2 u^2 of the sum) or as a tree of depth <= 12 (tensor-core rows,
// warp lanes): 12u; the division by m is correctly rounded: 1u.  Total
// (38 + 6 ln m) u + 2 L^2 u^2, doubled for the estimates above.
__host__ __device__ inline double f32_rel_bound(int k, int64_t m)
{
    const double u = 5.9604644775390625e-8;
    int64_t cells = 1;
    for (int t = 0; t < k; t++) cells *= 3;
    const double L = 2.0 * (double)cells;
    const double lnm = log((double)(m > 2 ? m : 2));
    return 2.0 * ((38.0 + 6.0 * lnm) * u + 2.0 * L * L * u * u);
}

// ---------------------------------------------------------------------------
// Candidate lists: (score, rank) pairs ordered by score descending, then
// rank ascending.  Kept in shared memory as separate arrays.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cand_better(float sa, uint64_t ra, float sb, uint64_t rb)
{
    return sa > sb || (sa == sb && ra < rb);
}

// Bitonic sort of size p2 (power of two) over the whole block.  Entries past
// the live count must already hold the sentinel (-1, ~0).
__device__ inline void block_sort_cands(float *sc, uint64_t *rk, int p2)
{
    for (int kk = 2; kk <= p2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
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
            __syncthreads();
        }
    }
}

__host__ __device__ inline int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace epi
