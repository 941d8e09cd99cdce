// Learned order-5 proposer: kernels and C-ABI.
//
// An exhaustive order-5 search is out of reach for large SNP counts (C(2000,5)
// = 2.65e14).  The proposer ranks candidate 5-sets with a small MLP fed by the
// lower-order scores of the candidate's SNPs (5 per-SNP, 10 pair and 10
// three-way MI values, and optionally the 5 four-way values, each group sorted
// so the features do not depend on SNP order); the best-ranked candidates are
// then recounted and scored exactly by the search's own kernels.  The network
// is trained on exhaustive order-5 scores of smaller instances.  Everything
// here runs in these kernels:
//   * features5_kernel: gathers and sorts the 25 (or 30) lower-order scores;
//   * gemm_kernel: C = A x B with FP32 accumulation over BF16 or FP32
//     operands in shared-memory tiles (every layer, forward and backward);
//   * bias/ReLU/convert, MSE-loss, column-sum and AdamW kernels;
//   * candidates5_kernel / cand_features5_kernel: the 5-sets made of a given
//     triple plus any two other SNPs, with their features.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "epi_host.h"
#include "epi_internal.cuh"

namespace epi {

void set_last_error(const char *msg);

namespace learn {

// ----------------------------------------------------------------- features
__device__ __forceinline__ uint64_t lex_rank(const uint64_t *tab, int64_t n, int k, const int32_t *c)
{
    uint64_t s = 0;
    for (int t = 0; t < k; t++) s += binom_at(tab, n, n - 1 - c[t], k - t);
    return binom_at(tab, n, n, k) - 1 - s;
}

// feature value of a score: ln(max(s, 0) + 1e-7) by the hardware log2
// approximation (about 2^-21 relative; the features only rank candidates)
__device__ __forceinline__ float feat_log(float s) { return __logf(fmaxf(s, 0.0f) + 1e-7f); }

template <int L>
__device__ __forceinline__ void sort_desc(float (&v)[L])
{
#pragma unroll
    for (int i = 1; i < L; i++) {
#pragma unroll
        for (int j = i; j > 0; j--) {
            const float a = v[j - 1], b = v[j];
            v[j - 1] = fmaxf(a, b);
            v[j] = fminf(a, b);
        }
    }
}

// 25 features of each 5-set: ln(MI + 1e-7) of its SNPs, pairs and triples,
// each group sorted descending; with the order-4 table s4, 30 features (the
// five four-way subsets' values appended, sorted descending).
__global__ void features5_kernel(DevData d, const float *__restrict__ s1, const float *__restrict__ s2,
                                 const float *__restrict__ s3, const float *__restrict__ s4,
                                 const uint32_t *__restrict__ combs, int64_t count, float *__restrict__ X)
{
    const int cols = s4 ? 30 : 25;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[5];
#pragma unroll
        for (int t = 0; t < 5; t++) c[t] = (int32_t)combs[i * 5 + t];
        float f1[5], f2[10], f3[10];
#pragma unroll
        for (int t = 0; t < 5; t++) f1[t] = s1[c[t]];
        int q = 0;
#pragma unroll
        for (int a = 0; a < 5; a++)
#pragma unroll
            for (int b = a + 1; b < 5; b++) {
                const int32_t p[2] = {c[a], c[b]};
                f2[q++] = s2[lex_rank(d.binom, d.n, 2, p)];
            }
        q = 0;
#pragma unroll
        for (int a = 0; a < 5; a++)
#pragma unroll
            for (int b = a + 1; b < 5; b++)
#pragma unroll
                for (int e = b + 1; e < 5; e++) {
                    const int32_t p[3] = {c[a], c[b], c[e]};
                    f3[q++] = s3[lex_rank(d.binom, d.n, 3, p)];
                }
        sort_desc(f1);
        sort_desc(f2);
        sort_desc(f3);
        float *x = X + i * cols;
#pragma unroll
        for (int t = 0; t < 5; t++) x[t] = feat_log(f1[t]);
#pragma unroll
        for (int t = 0; t < 10; t++) x[5 + t] = feat_log(f2[t]);
#pragma unroll
        for (int t = 0; t < 10; t++) x[15 + t] = feat_log(f3[t]);
        if (s4) {
            float f4[5];
#pragma unroll
            for (int j = 0; j < 5; j++) {
                int32_t p[4];
                int m = 0;
#pragma unroll
                for (int t = 0; t < 5; t++)
                    if (t != j) p[m++] = c[t];
                f4[j] = s4[lex_rank(d.binom, d.n, 4, p)];
            }
            sort_desc(f4);
#pragma unroll
            for (int t = 0; t < 5; t++) x[25 + t] = feat_log(f4[t]);
        }
    }
}

// 5-set number g of the space made of triple T[t] and two other SNPs u < v
// (any order relative to the triple), enumerated as g = t * C(n-3, 2) + (lex
// rank of (u, v) among the other n-3 SNPs).  v[] receives the sorted set,
// g3[] the generating triple.
__device__ __forceinline__ void candidate_at(const DevData &d, const uint32_t *__restrict__ triples, uint64_t g,
                                             int32_t (&v)[5], int32_t (&g3)[3])
{
    const int64_t rest = d.n - 3;
    const uint64_t per = (uint64_t)(rest * (rest - 1) / 2);
    const uint64_t t = (g >> 32) == 0 && (per >> 32) == 0 ? (uint64_t)((uint32_t)g / (uint32_t)per) : g / per;
    const int64_t r = (int64_t)(g - t * per);
    const int32_t a = (int32_t)triples[t * 3], b = (int32_t)triples[t * 3 + 1], c = (int32_t)triples[t * 3 + 2];
    g3[0] = a; g3[1] = b; g3[2] = c;
    // pair (x, y) of [0, rest) with lexicographic rank r: pairs whose first
    // element is below x number S(x) = x (2 rest - x - 1) / 2; x is the
    // largest value with S(x) <= r (closed form in single precision, then
    // corrected by integer comparisons)
    auto S = [&](int64_t x) { return x * (2 * rest - x - 1) / 2; };
    const float B = (float)(2 * rest - 1);
    int64_t x = (int64_t)((B - sqrtf(fmaxf(B * B - 8.0f * (float)r, 0.0f))) * 0.5f);
    if (x < 0) x = 0;
    if (x > rest - 2) x = rest - 2;
    while (x > 0 && S(x) > r) x--;
    while (x < rest - 2 && S(x + 1) <= r) x++;
    const int64_t y = x + 1 + (r - S(x));
    // map indices of [0, rest) to SNPs other than a, b, c
    auto skip = [&](int64_t z) {
        int64_t s = z;
        if (s >= a) s++;
        if (s >= b) s++;
        if (s >= c) s++;
        return (int32_t)s;
    };
    v[0] = a; v[1] = b; v[2] = c; v[3] = skip(x); v[4] = skip(y);
#pragma unroll
    for (int p = 1; p < 5; p++)
#pragma unroll
        for (int q = p; q > 0; q--) {
            const int32_t lo = min(v[q - 1], v[q]), hi = max(v[q - 1], v[q]);
            v[q - 1] = lo;
            v[q] = hi;
        }
}

// Whether the generating triple g3 is the best of the set's ten triples by
// (order-3 score desc, rank asc): a set holding several listed triples is
// then kept once, under the best of them.
__device__ __forceinline__ bool generated_by_best(const DevData &d, const float *__restrict__ s3, const int32_t (&v)[5],
                                                  const int32_t (&g3)[3])
{
    const uint64_t gr = lex_rank(d.binom, d.n, 3, g3);
    const float gs = s3[gr];
    bool best = true;
#pragma unroll
    for (int x1 = 0; x1 < 5; x1++)
#pragma unroll
        for (int x2 = x1 + 1; x2 < 5; x2++)
#pragma unroll
            for (int x3 = x2 + 1; x3 < 5; x3++) {
                const int32_t p[3] = {v[x1], v[x2], v[x3]};
                const uint64_t r3 = lex_rank(d.binom, d.n, 3, p);
                const float sc = s3[r3];
                if (sc > gs || (sc == gs && r3 < gr)) best = false;
            }
    return best;
}

// candidates [first, first + count) of the triples-plus-pair space
__global__ void candidates5_kernel(DevData d, const uint32_t *__restrict__ triples, int64_t first, int64_t count,
                                   uint32_t *__restrict__ combs, const float *__restrict__ s3, uint8_t *__restrict__ keep)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[5], g3[3];
        candidate_at(d, triples, (uint64_t)(first + i), v, g3);
#pragma unroll
        for (int p = 0; p < 5; p++) combs[i * 5 + p] = (uint32_t)v[p];
        if (keep) keep[i] = generated_by_best(d, s3, v, g3) ? 1 : 0;
    }
}

// candidates at listed indices of the same space
__global__ void candidates5_at_kernel(DevData d, const uint32_t *__restrict__ triples, const uint64_t *__restrict__ idx,
                                      int64_t count, uint32_t *__restrict__ combs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[5], g3[3];
        candidate_at(d, triples, idx[i], v, g3);
#pragma unroll
        for (int p = 0; p < 5; p++) combs[i * 5 + p] = (uint32_t)v[p];
    }
}

// Candidates [first, first + count) in one pass: the set, whether its
// generating triple is its best (keep) and its 25 features (30 with the
// order-4 table s4); the set itself is written only when combs is given.
constexpr int kFeatThreads = 256;

__global__ void __launch_bounds__(kFeatThreads) cand_features5_kernel(DevData d, const uint32_t *__restrict__ triples,
                                                             int64_t first, int64_t count, const float *__restrict__ s1,
                                                             const float *__restrict__ s2, const float *__restrict__ s3,
                                                             const float *__restrict__ s4, float *__restrict__ X,
                                                             uint8_t *__restrict__ keep, uint32_t *__restrict__ combs)
{
    const int64_t n = d.n;
    const int cols = s4 ? 30 : 25;
    const int stride = cols | 1;          // odd row stride in shared memory: no bank conflicts
    // a block's rows are staged here and written out coalesced (each thread
    // owning a 100- or 120-byte row would scatter every store over 32 rows)
    __shared__ float rows_s[kFeatThreads * 31];
    // binomials C(x, 2), C(x, 3), C(x, 4) from the dataset's table (L1-resident rows)
    const uint64_t *__restrict__ b2 = d.binom + 2 * (n + 1);
    const uint64_t *__restrict__ b3 = d.binom + 3 * (n + 1);
    const uint64_t *__restrict__ b4 = d.binom + 4 * (n + 1);
    const uint64_t n2 = b2[n], n3 = b3[n];
    for (int64_t base = (int64_t)blockIdx.x * kFeatThreads; base < count; base += (int64_t)gridDim.x * kFeatThreads) {
        const int64_t i = base + threadIdx.x;
        const int nrows = count - base < kFeatThreads ? (int)(count - base) : kFeatThreads;
        __syncthreads();                  // the previous rows are written out
        if (i < count) {
        int32_t v[5], g3[3];
        candidate_at(d, triples, (uint64_t)(first + i), v, g3);
        if (combs) {
#pragma unroll
            for (int p = 0; p < 5; p++) combs[i * 5 + p] = (uint32_t)v[p];
        }
        // the ten triples: ranks and scores; the generating triple's rank
        const uint64_t gr = n3 - 1 - (b3[n - 1 - g3[0]] + b2[n - 1 - g3[1]] + (uint64_t)(n - 1 - g3[2]));
        float f3[10];
        float gs = 0.0f;
        uint64_t r3[10];
        int q = 0;
#pragma unroll
        for (int a = 0; a < 5; a++)
#pragma unroll
            for (int b = a + 1; b < 5; b++)
#pragma unroll
                for (int e = b + 1; e < 5; e++) {
                    r3[q] = n3 - 1 - (b3[n - 1 - v[a]] + b2[n - 1 - v[b]] + (uint64_t)(n - 1 - v[e]));
                    f3[q] = s3[r3[q]];
                    if (r3[q] == gr) gs = f3[q];
                    q++;
                }
        bool best = true;
#pragma unroll
        for (int t = 0; t < 10; t++)
            if (f3[t] > gs || (f3[t] == gs && r3[t] < gr)) best = false;
        keep[i] = best ? 1 : 0;
        float f2[10], f1[5];
        q = 0;
#pragma unroll
        for (int a = 0; a < 5; a++)
#pragma unroll
            for (int b = a + 1; b < 5; b++) f2[q++] = s2[n2 - 1 - (b2[n - 1 - v[a]] + (uint64_t)(n - 1 - v[b]))];
#pragma unroll
        for (int t = 0; t < 5; t++) f1[t] = s1[v[t]];
        sort_desc(f1);
        sort_desc(f2);
        sort_desc(f3);
        float *x = rows_s + threadIdx.x * stride;
#pragma unroll
        for (int t = 0; t < 5; t++) x[t] = feat_log(f1[t]);
#pragma unroll
        for (int t = 0; t < 10; t++) x[5 + t] = feat_log(f2[t]);
#pragma unroll
        for (int t = 0; t < 10; t++) x[15 + t] = feat_log(f3[t]);
        if (s4) {
            // the five four-way subsets (v sorted ascending): drop v[j]
            const uint64_t n4 = b4[n];
            float f4[5];
#pragma unroll
            for (int j = 0; j < 5; j++) {
                int32_t p[4];
                int m = 0;
#pragma unroll
                for (int t = 0; t < 5; t++)
                    if (t != j) p[m++] = v[t];
                const uint64_t r4 = n4 - 1 - (b4[n - 1 - p[0]] + b3[n - 1 - p[1]] + b2[n - 1 - p[2]] +
                                              (uint64_t)(n - 1 - p[3]));
                f4[j] = s4[r4];
            }
            sort_desc(f4);
#pragma unroll
            for (int t = 0; t < 5; t++) x[25 + t] = feat_log(f4[t]);
        }
        }
        __syncthreads();
        // the block's rows are contiguous in X: coalesced word stores
        float *dst = X + base * cols;
        const int words = nrows * cols;
        for (int w = threadIdx.x; w < words; w += kFeatThreads) {
            const int row = w / cols, col = w - row * cols;
            dst[w] = rows_s[row * stride + col];
        }
    }
}

// out[i] = table[lex rank of combs[i]] for an order-k score table
__global__ void lookup_kernel(DevData d, int k, const float *__restrict__ table, const uint32_t *__restrict__ combs,
                              int64_t count, float *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[EPI_MAX_ORDER];
        for (int t = 0; t < k; t++) c[t] = (int32_t)combs[i * k + t];
        out[i] = table[lex_rank(d.binom, d.n, k, c)];
    }
}

// --------------------------------------------------------------------- MLP
// C[M x N] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m * sam + k * sak], etc.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const TA *__restrict__ A, int64_t sam,
                                                   int64_t sak, const TB *__restrict__ B, int64_t sbk, int64_t sbn,
                                                   float *__restrict__ C, int64_t scm, int64_t scn, int accumulate)
{
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;   // rows on x: no 65535 limit
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e >> 6, mm = e & 63;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? (float)A[(int64_t)m * sam + (int64_t)k * sak] : 0.0f;
            const int n = n0 + mm;
            Bs[kk][mm] = (n < N && k < K) ? (float)B[(int64_t)k * sbk + (int64_t)n * sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float *o = C + (int64_t)m * scm + (int64_t)n * scn;
                *o = accumulate ? *o + acc[i][j] : acc[i][j];
            }
        }
}

// Z[B x N] fp32 + bias -> optional ReLU -> BF16 activations (and FP32 copy)
__global__ void bias_act_kernel(const float *__restrict__ Z, const float *__restrict__ bias, int64_t rows, int N, int relu,
                                __nv_bfloat16 *__restrict__ H, float *__restrict__ Hf)
{
    const int64_t total = rows * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        float v = Z[i] + bias[i % N];
        if (relu) v = fmaxf(v, 0.0f);
        if (H) H[i] = __float2bfloat16(v);
        if (Hf) Hf[i] = v;
    }
}

// network input: (X - shift) * scale per feature, to BF16
__global__ void input_kernel(const float *__restrict__ X, int64_t rows, int n_in, const float *__restrict__ norm,
                             __nv_bfloat16 *__restrict__ Y)
{
    const int64_t total = rows * n_in;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i % n_in);
        Y[i] = __float2bfloat16((X[i] - norm[f]) * norm[n_in + f]);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ X, int64_t total, __nv_bfloat16 *__restrict__ Y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        Y[i] = __float2bfloat16(X[i]);
}

// dY = 2 (y - t) / B, and the summed squared error
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ t, int64_t rows, float *__restrict__ dy,
                           float *__restrict__ loss)
{
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        dy[i] = 2.0f * e / (float)rows;
        acc += e * e;
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (float)rows);
}

// dZ = dH * (H > 0) (in place on dH, ReLU derivative from the activations)
__global__ void relu_grad_kernel(float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H, int64_t total)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(H[i]) > 0.0f)) dH[i] = 0.0f;
}

// db[n] = sum over rows of dZ[row][n]
__global__ void colsum_kernel(const float *__restrict__ dZ, int64_t rows, int N, float *__restrict__ db)
{
    const int n = blockIdx.x;
    float acc = 0.0f;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += dZ[r * N + n];
    __shared__ float part[256];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[n] = part[0];
}

// Reductions over the batch, sliced: part[s][i][j] = sum over the rows b of
// slice s of U[b][i] V[b][j] for j < nj, and part[s][i][nj] = sum of U[b][i]
// (the bias gradient); one thread per i, the slice's V rows staged in shared
// memory.  Slices of kSliceRows rows keep every CTA busy whatever the batch.
constexpr int kSliceRows = 64;
constexpr int kMaxNj = 32;

template <typename TU, typename TV>
__global__ void __launch_bounds__(256) batch_outer_kernel(const TU *__restrict__ U, int64_t ldu,
                                                          const TV *__restrict__ V, int64_t ldv, int64_t B, int ni,
                                                          int nj, float *__restrict__ part)
{
    __shared__ float vs[kSliceRows][kMaxNj];
    const int64_t b0 = (int64_t)blockIdx.x * kSliceRows;
    const int rows = (int)min((int64_t)kSliceRows, B - b0);
    for (int e = threadIdx.x; e < rows * nj; e += blockDim.x) {
        const int r = e / nj, j = e - r * nj;
        vs[r][j] = (float)V[(b0 + r) * ldv + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ni; i += blockDim.x) {
        float acc[kMaxNj];
#pragma unroll
        for (int j = 0; j < kMaxNj; j++) acc[j] = 0.0f;
        float bias = 0.0f;
        for (int r = 0; r < rows; r++) {
            const float u = (float)U[(b0 + r) * ldu + i];
            bias += u;
#pragma unroll
            for (int j = 0; j < kMaxNj; j++)
                if (j < nj) acc[j] = fmaf(u, vs[r][j], acc[j]);
        }
        float *o = part + ((size_t)blockIdx.x * ni + i) * (nj + 1);
        for (int j = 0; j < nj; j++) o[j] = acc[j];
        o[nj] = bias;
    }
}

// G[i][j] = sum over the slices (in slice order) of part[s][i][j], and the
// bias sums into gb[i] (either output may be NULL)
__global__ void sum_outer_kernel(const float *__restrict__ part, int slices, int ni, int nj, float *__restrict__ G,
                                 float *__restrict__ gb)
{
    const int per = nj + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ni * per; e += gridDim.x * blockDim.x) {
        float sum = 0.0f;
        for (int q = 0; q < slices; q++) sum += part[(size_t)q * ni * per + e];
        const int i = e / per, j = e - i * per;
        if (j < nj) { if (G) G[i * nj + j] = sum; }
        else if (gb) gb[i] = sum;
    }
}

// Tiled transpose into BF16: out[c][r] = in[r][c] for r < R, c < C (rows of
// `in` ld_in apart, of `out` ld_out apart); optionally also the same values
// in BF16 without transposing (out_same[r][c], stride C).
template <typename T>
__global__ void transpose_bf16_kernel(const T *__restrict__ in, int64_t R, int C, int64_t ld_in,
                                      __nv_bfloat16 *__restrict__ out, int64_t ld_out,
                                      __nv_bfloat16 *__restrict__ out_same)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (r < R && c < C) {
            v = __float2bfloat16((float)in[r * ld_in + c]);
            if (out_same) out_same[r * C + c] = v;
        }
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (c < C && r < R) out[(int64_t)c * ld_out + r] = tile[threadIdx.x][i];
    }
}

// AdamW on the FP32 master weights; BF16 working copies refreshed
__global__ void adamw_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                             float *__restrict__ m2, __nv_bfloat16 *__restrict__ wb, int64_t count, float lr, float b1,
                             float b2, float eps, float wd, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        const float mh = a / c1, vh = v / c2;
        float wi = w[i];
        wi -= lr * (mh / (sqrtf(vh) + eps) + wd * wi);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

// The ranking without the network: the sum of the ten three-way log-scores
// of 25-column rows, or of the five four-way log-scores of 30-column rows.
__global__ void heuristic5_kernel(const float *__restrict__ X, int64_t count, int cols, float *__restrict__ out)
{
    const int lo = cols == 30 ? 25 : 15;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int t = lo; t < cols; t++) s += X[i * cols + t];
        out[i] = s;
    }
}

}  // namespace learn

// candidate-list comparison for the top-k: -inf below any real score
}  // namespace epi

// ===================================================================== API
using namespace epi;

struct epi_mlp {
    int n_in = 25, hidden = 256;
    int64_t n_params = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    float *w = nullptr;            // FP32 master weights: W1 [h][in], b1 [h], W2 [h][h], b2 [h], W3 [1][h], b3 [1]
    float *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wb = nullptr;   // BF16 working copy
    float *norm = nullptr;         // input shift [n_in] then scale [n_in]
    int32_t *status = nullptr;     // tensor-core inference status word
    int forward_path = 0;          // 0 auto, 1 CUDA cores, 2 tensor cores
    int num_sms = 0;
    int64_t step = 0;
    // activation buffers for a batch (grown on demand)
    int64_t cap = 0;
    void *act = nullptr;
};

namespace {

epi_status lfail(epi_status s, const char *msg)
{
    epi::set_last_error(msg);
    return s;
}

#define LCK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return lfail(EPI_ECUDA, cudaGetErrorString(e_));     \
    } while (0)

struct Offs {
    int64_t W1, b1, W2, b2, W3, b3, total;
};

Offs offsets(int in, int h)
{
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)h * in;
    o.W2 = o.b1 + h;
    o.b2 = o.W2 + (int64_t)h * h;
    o.W3 = o.b2 + h;
    o.b3 = o.W3 + h;
    o.total = o.b3 + 1;
    return o;
}

int blocks_for(int64_t n, int per = 256) { return (int)std::min<int64_t>((n + per - 1) / per, 4096); }

template <typename TA, typename TB>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const TA *A, int64_t sam, int64_t sak, const TB *B, int64_t sbk,
                 int64_t sbn, float *C, int64_t scm, int64_t scn, int accumulate)
{
    dim3 grid((M + 63) / 64, (N + 63) / 64);
    learn::gemm_kernel<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, scm, scn, accumulate);
    return cudaGetLastError();
}

// activation layout of a batch of B rows
struct Acts {
    __nv_bfloat16 *X;    // [B][in]
    float *Z1;           // [B][h] pre-activations, reused for gradients
    __nv_bfloat16 *H1;   // [B][h]
    float *Z2;
    __nv_bfloat16 *H2;
    float *Y;            // [B]
    float *dY;           // [B]
    float *loss;         // [1]
    // tensor-core products of the training step (hidden a multiple of 8)
    int64_t Bp;          // B rounded up to a multiple of 8 (row stride of the transposes)
    __nv_bfloat16 *H1t;  // [h][Bp]  H1 transposed
    __nv_bfloat16 *dZb;  // [B][h]   dZ2 in BF16
    __nv_bfloat16 *dZt;  // [h][Bp]  dZ2 in BF16, transposed
    __nv_bfloat16 *W2t;  // [h][h]   W2 transposed (BF16 working copy)
    float *part;         // split-K partial tiles of dW2
    float *opart;        // [slices][h][n_in + 1] partial sums of the batch reductions
};

// The three hidden x hidden products of a training step run on the tensor
// cores (epi_gemm_tc.cu) when the hidden width allows 16-byte rows.
bool train_tc(const epi_mlp *net);

epi_status ensure_acts(epi_mlp *net, int64_t B, Acts &a)
{
    const int in = net->n_in, h = net->hidden;
    auto bytes = [&](int64_t rows) {
        const int64_t rp = (rows + 7) / 8 * 8;
        size_t b = (size_t)rows * in * 2 + (size_t)rows * h * 4 * 2 + (size_t)rows * h * 2 * 2 + (size_t)rows * 8 + 1024 +
                   6 * 256;
        if (train_tc(net))
            b += (size_t)h * rp * 2 * 2 + (size_t)rows * h * 2 + (size_t)h * h * 2 +
                 gemm_tc_partial_floats(h, h, (int)std::min<int64_t>(rows, INT32_MAX), net->num_sms) * 4 + 5 * 256;
        b += (size_t)((rows + learn::kSliceRows - 1) / learn::kSliceRows) * h * (std::max(in, 1) + 1) * 4 + 256;
        return b;
    };
    if (net->cap < B) {
        if (net->act) cudaFree(net->act);
        net->act = nullptr;
        net->cap = 0;
        LCK(cudaMalloc(&net->act, bytes(B)));
        net->cap = B;
    }
    char *p = static_cast<char *>(net->act);
    auto take = [&](size_t n) { char *r = p; p += (n + 255) & ~(size_t)255; return r; };
    a.X = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * in * 2));
    a.Z1 = reinterpret_cast<float *>(take((size_t)B * h * 4));
    a.H1 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * h * 2));
    a.Z2 = reinterpret_cast<float *>(take((size_t)B * h * 4));
    a.H2 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * h * 2));
    a.Y = reinterpret_cast<float *>(take((size_t)B * 4));
    a.dY = reinterpret_cast<float *>(take((size_t)B * 4));
    a.loss = reinterpret_cast<float *>(take(4));
    a.Bp = (B + 7) / 8 * 8;
    a.H1t = a.dZb = a.dZt = a.W2t = nullptr;
    a.part = nullptr;
    if (train_tc(net)) {
        a.H1t = reinterpret_cast<__nv_bfloat16 *>(take((size_t)h * a.Bp * 2));
        a.dZt = reinterpret_cast<__nv_bfloat16 *>(take((size_t)h * a.Bp * 2));
        a.dZb = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * h * 2));
        a.W2t = reinterpret_cast<__nv_bfloat16 *>(take((size_t)h * h * 2));
        a.part = reinterpret_cast<float *>(take(gemm_tc_partial_floats(h, h, (int)B, net->num_sms) * 4));
    }
    a.opart = reinterpret_cast<float *>(
        take((size_t)((B + learn::kSliceRows - 1) / learn::kSliceRows) * h * (std::max(in, 1) + 1) * 4));
    return EPI_OK;
}

bool train_tc(const epi_mlp *net) { return net->hidden % 8 == 0; }

template <typename T>
cudaError_t transpose_bf16(const T *in, int64_t R, int C, int64_t ld_in, __nv_bfloat16 *out, int64_t ld_out,
                           __nv_bfloat16 *out_same, cudaStream_t st)
{
    dim3 grid((unsigned)((R + 31) / 32), (unsigned)((C + 31) / 32));
    learn::transpose_bf16_kernel<T><<<grid, dim3(32, 8), 0, st>>>(in, R, C, ld_in, out, ld_out, out_same);
    return cudaGetLastError();
}

// tc: the layer-2 product on the tensor cores (training); otherwise every
// layer on the CUDA cores
epi_status forward(epi_mlp *net, const float *X, int64_t B, Acts &a, float *y_out, bool tc = false)
{
    const int in = net->n_in, h = net->hidden;
    const Offs o = offsets(in, h);
    cudaStream_t st = net->stream;
    learn::input_kernel<<<blocks_for(B * in), 256, 0, st>>>(X, B, in, net->norm, a.X);
    // layer 1: Z1 = X W1^T, H1 = relu(Z1 + b1)
    LCK(gemm(st, (int)B, h, in, a.X, in, 1, net->wb + o.W1, 1, in, a.Z1, h, 1, 0));
    learn::bias_act_kernel<<<blocks_for(B * h), 256, 0, st>>>(a.Z1, net->w + o.b1, B, h, 1, a.H1, nullptr);
    if (tc && train_tc(net))
        LCK(launch_gemm_tc(a.H1, h, net->wb + o.W2, h, a.Z2, h, (int)B, h, h, nullptr, net->status, net->num_sms, st));
    else
        LCK(gemm(st, (int)B, h, h, a.H1, h, 1, net->wb + o.W2, 1, h, a.Z2, h, 1, 0));
    learn::bias_act_kernel<<<blocks_for(B * h), 256, 0, st>>>(a.Z2, net->w + o.b2, B, h, 1, a.H2, nullptr);
    LCK(gemm(st, (int)B, 1, h, a.H2, h, 1, net->wb + o.W3, 1, h, y_out, 1, 1, 0));
    learn::bias_act_kernel<<<blocks_for(B), 256, 0, st>>>(y_out, net->w + o.b3, B, 1, 0, nullptr, y_out);
    return EPI_OK;
}

// gradients of the mean squared error into net->g; loss (device) summed in a.loss
epi_status backward(epi_mlp *net, const float *t, int64_t B, Acts &a)
{
    const int in = net->n_in, h = net->hidden;
    const Offs o = offsets(in, h);
    cudaStream_t st = net->stream;
    LCK(cudaMemsetAsync(a.loss, 0, 4, st));
    learn::mse_kernel<<<blocks_for(B), 256, 0, st>>>(a.Y, t, B, a.dY, a.loss);
    // layer 3: dW3 = dY^T H2, db3 = sum dY, dH2 = dY W3
    const int slices = (int)((B + learn::kSliceRows - 1) / learn::kSliceRows);
    auto sum_outer = [&](int ni, int nj, float *G, float *gb) {
        const int total = ni * (nj + 1);
        learn::sum_outer_kernel<<<(total + 255) / 256, 256, 0, st>>>(a.opart, slices, ni, nj, G, gb);
        return cudaGetLastError();
    };
    learn::batch_outer_kernel<<<slices, 256, 0, st>>>(a.H2, h, a.dY, 1, B, h, 1, a.opart);
    LCK(sum_outer(h, 1, net->g + o.W3, nullptr));
    learn::colsum_kernel<<<1, 256, 0, st>>>(a.dY, B, 1, net->g + o.b3);
    float *dZ2 = a.Z2;   // reuse
    LCK(gemm(st, (int)B, h, 1, a.dY, 1, 1, net->wb + o.W3, 1, 1, dZ2, h, 1, 0));
    learn::relu_grad_kernel<<<blocks_for(B * h), 256, 0, st>>>(dZ2, a.H2, B * h);
    float *dZ1 = a.Z1;
    if (train_tc(net)) {
        // layer 2 on the tensor cores: dZ2 in BF16 (row-major and
        // transposed), H1 and W2 transposed, so both products are K-major
        LCK(transpose_bf16(a.H1, B, h, h, a.H1t, a.Bp, nullptr, st));
        LCK(transpose_bf16(dZ2, B, h, h, a.dZt, a.Bp, a.dZb, st));
        LCK(transpose_bf16(net->wb + o.W2, h, h, h, a.W2t, h, nullptr, st));
        // dW2 = dZ2^T H1 (K = the batch, split over CTAs), db2, dH1 = dZ2 W2
        LCK(launch_gemm_tc(a.dZt, a.Bp, a.H1t, a.Bp, net->g + o.W2, h, h, h, (int)B, a.part, net->status, net->num_sms,
                           st));
        learn::batch_outer_kernel<<<slices, 256, 0, st>>>(dZ2, h, a.X, in, B, h, 0, a.opart);
        LCK(sum_outer(h, 0, nullptr, net->g + o.b2));
        LCK(launch_gemm_tc(a.dZb, h, a.W2t, h, dZ1, h, (int)B, h, h, nullptr, net->status, net->num_sms, st));
    } else {
        // layer 2: dW2 = dZ2^T H1, db2, dH1 = dZ2 W2
        LCK(gemm(st, h, h, (int)B, dZ2, 1, h, a.H1, h, 1, net->g + o.W2, h, 1, 0));
        learn::colsum_kernel<<<h, 256, 0, st>>>(dZ2, B, h, net->g + o.b2);
        LCK(gemm(st, (int)B, h, h, dZ2, h, 1, net->wb + o.W2, h, 1, dZ1, h, 1, 0));
    }
    learn::relu_grad_kernel<<<blocks_for(B * h), 256, 0, st>>>(dZ1, a.H1, B * h);
    // layer 1: dW1 = dZ1^T X, db1 (sliced over the batch for up to 32 inputs)
    if (in <= learn::kMaxNj) {
        learn::batch_outer_kernel<<<slices, 256, 0, st>>>(dZ1, h, a.X, in, B, h, in, a.opart);
        LCK(sum_outer(h, in, net->g + o.W1, net->g + o.b1));
    } else {
        LCK(gemm(st, h, in, (int)B, dZ1, 1, h, a.X, in, 1, net->g + o.W1, in, 1, 0));
        learn::colsum_kernel<<<h, 256, 0, st>>>(dZ1, B, h, net->g + o.b1);
    }
    return EPI_OK;
}

}  // namespace

extern "C" {

epi_status epi_mlp_create(epi_ctx *ctx, int n_in, int hidden, uint64_t seed, epi_mlp **out)
{
    if (!ctx || !out) return lfail(EPI_EINVAL, "NULL argument");
    if (n_in < 1 || n_in > 1024 || hidden < 1 || hidden > 4096)
        return lfail(EPI_EINVAL, "epi_mlp_create: n_in in 1..1024, hidden in 1..4096");
    epi_mlp *net = new epi_mlp();
    net->n_in = n_in;
    net->hidden = hidden;
    net->stream = epi_ctx_stream(ctx);
    net->device = epi_ctx_device(ctx);
    net->num_sms = epi_ctx_num_sms(ctx);
    cudaSetDevice(net->device);
    const Offs o = offsets(n_in, hidden);
    net->n_params = o.total;
    const size_t fb = (size_t)o.total * 4;
    if (cudaMalloc((void **)&net->w, fb) != cudaSuccess || cudaMalloc((void **)&net->g, fb) != cudaSuccess ||
        cudaMalloc((void **)&net->m1, fb) != cudaSuccess || cudaMalloc((void **)&net->m2, fb) != cudaSuccess ||
        cudaMalloc((void **)&net->wb, (size_t)o.total * 2) != cudaSuccess ||
        cudaMalloc((void **)&net->norm, (size_t)n_in * 8) != cudaSuccess ||
        cudaMalloc((void **)&net->status, 4) != cudaSuccess) {
        epi_mlp_destroy(net);
        return lfail(EPI_ENOMEM, "epi_mlp_create: allocation failed");
    }
    // He-uniform initialisation from SplitMix64 draws (host), biases 0
    std::vector<float> h((size_t)o.total, 0.0f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        const double lim = std::sqrt(6.0 / (double)fan_in);
        for (int64_t i = 0; i < count; i++) h[(size_t)(off + i)] = (float)((2.0 * next() - 1.0) * lim);
    };
    fill(o.W1, (int64_t)hidden * n_in, n_in);
    fill(o.W2, (int64_t)hidden * hidden, hidden);
    fill(o.W3, hidden, hidden);
    epi_status s = epi_mlp_set_params(net, h.data());
    if (s == EPI_OK) {
        std::vector<float> nm((size_t)n_in * 2, 0.0f);
        for (int f = 0; f < n_in; f++) nm[(size_t)n_in + f] = 1.0f;
        s = epi_mlp_set_input_norm(net, nm.data(), nm.data() + n_in);
    }
    if (s != EPI_OK) { epi_mlp_destroy(net); return s; }
    cudaMemsetAsync(net->m1, 0, fb, net->stream);
    cudaMemsetAsync(net->m2, 0, fb, net->stream);
    *out = net;
    return EPI_OK;
}

void epi_mlp_destroy(epi_mlp *net)
{
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    cudaFree(net->w); cudaFree(net->g); cudaFree(net->m1); cudaFree(net->m2); cudaFree(net->wb); cudaFree(net->norm); cudaFree(net->status);
    if (net->act) cudaFree(net->act);
    delete net;
}

int64_t epi_mlp_num_params(const epi_mlp *net) { return net ? net->n_params : 0; }
int epi_mlp_num_inputs(const epi_mlp *net) { return net ? net->n_in : 0; }

epi_status epi_mlp_get_params(const epi_mlp *net, float *host)
{
    if (!net || !host) return lfail(EPI_EINVAL, "NULL argument");
    LCK(cudaMemcpyAsync(host, net->w, (size_t)net->n_params * 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaStreamSynchronize(net->stream));
    return EPI_OK;
}

epi_status epi_mlp_set_params(epi_mlp *net, const float *host)
{
    if (!net || !host) return lfail(EPI_EINVAL, "NULL argument");
    LCK(cudaMemcpyAsync(net->w, host, (size_t)net->n_params * 4, cudaMemcpyHostToDevice, net->stream));
    learn::to_bf16_kernel<<<blocks_for(net->n_params), 256, 0, net->stream>>>(net->w, net->n_params, net->wb);
    LCK(cudaGetLastError());
    LCK(cudaStreamSynchronize(net->stream));
    net->step = 0;
    return EPI_OK;
}

epi_status epi_mlp_set_input_norm(epi_mlp *net, const float *shift_host, const float *scale_host)
{
    if (!net || !shift_host || !scale_host) return lfail(EPI_EINVAL, "NULL argument");
    LCK(cudaMemcpyAsync(net->norm, shift_host, (size_t)net->n_in * 4, cudaMemcpyHostToDevice, net->stream));
    LCK(cudaMemcpyAsync(net->norm + net->n_in, scale_host, (size_t)net->n_in * 4, cudaMemcpyHostToDevice, net->stream));
    LCK(cudaStreamSynchronize(net->stream));
    return EPI_OK;
}

epi_status epi_mlp_get_input_norm(const epi_mlp *net, float *shift_host, float *scale_host)
{
    if (!net || !shift_host || !scale_host) return lfail(EPI_EINVAL, "NULL argument");
    LCK(cudaMemcpyAsync(shift_host, net->norm, (size_t)net->n_in * 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaMemcpyAsync(scale_host, net->norm + net->n_in, (size_t)net->n_in * 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaStreamSynchronize(net->stream));
    return EPI_OK;
}

epi_status epi_mlp_set_forward_path(epi_mlp *net, int path)
{
    if (!net || path < 0 || path > 2) return lfail(EPI_EINVAL, "epi_mlp_set_forward_path: bad argument");
    if (path == 2 && !mlp_tc_applies(net->n_in, net->hidden))
        return lfail(EPI_EUNSUPPORTED, "tensor-core inference needs hidden = 256 and n_in <= 32");
    net->forward_path = path;
    return EPI_OK;
}

epi_status epi_mlp_forward(epi_mlp *net, const float *X_dev, int64_t rows, float *y_dev)
{
    if (!net || !X_dev || !y_dev || rows < 1) return lfail(EPI_EINVAL, "epi_mlp_forward: bad argument");
    if (net->forward_path != 1 && mlp_tc_applies(net->n_in, net->hidden)) {
        const int in = net->n_in, h = net->hidden;
        const Offs o = offsets(in, h);
        LCK(cudaMemsetAsync(net->status, 0, 4, net->stream));
        LCK(launch_mlp_forward_tc(X_dev, rows, nullptr, nullptr, in, net->norm, net->wb + o.W1, net->w + o.b1,
                                  net->wb + o.W2, net->w + o.b2, net->wb + o.W3, net->w + o.b3, y_dev, net->status,
                                  net->num_sms, net->stream));
        int32_t st = 0;
        LCK(cudaMemcpyAsync(&st, net->status, 4, cudaMemcpyDeviceToHost, net->stream));
        LCK(cudaStreamSynchronize(net->stream));
        if (st) return lfail(EPI_ETIMEOUT, "epi_mlp_forward: a tensor-core wait gave up");
        return EPI_OK;
    }
    // slices of at most 128K rows bound the activation memory
    constexpr int64_t kSlice = (int64_t)1 << 17;
    Acts a;
    epi_status s = ensure_acts(net, std::min(rows, kSlice), a);
    for (int64_t r0 = 0; s == EPI_OK && r0 < rows; r0 += kSlice) {
        const int64_t nr = std::min(kSlice, rows - r0);
        s = forward(net, X_dev + r0 * net->n_in, nr, a, y_dev + r0);
    }
    return s;
}

epi_status epi_mlp_gradients(epi_mlp *net, const float *X_dev, const float *t_dev, int64_t rows, float *grad_host,
                             float *loss_host)
{
    if (!net || !X_dev || !t_dev || rows < 1) return lfail(EPI_EINVAL, "epi_mlp_gradients: bad argument");
    Acts a;
    epi_status s = ensure_acts(net, rows, a);
    if (s == EPI_OK) LCK(cudaMemsetAsync(net->status, 0, 4, net->stream));
    if (s == EPI_OK) s = forward(net, X_dev, rows, a, a.Y, true);
    if (s == EPI_OK) s = backward(net, t_dev, rows, a);
    if (s != EPI_OK) return s;
    int32_t hs = 0;
    if (grad_host) LCK(cudaMemcpyAsync(grad_host, net->g, (size_t)net->n_params * 4, cudaMemcpyDeviceToHost, net->stream));
    if (loss_host) LCK(cudaMemcpyAsync(loss_host, a.loss, 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaMemcpyAsync(&hs, net->status, 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaStreamSynchronize(net->stream));
    if (hs) return lfail(EPI_ETIMEOUT, "epi_mlp_gradients: a tensor-core wait gave up");
    return EPI_OK;
}

epi_status epi_mlp_train_step(epi_mlp *net, const float *X_dev, const float *t_dev, int64_t rows, float lr, float wd,
                              float *loss_host)
{
    if (!net || !X_dev || !t_dev || rows < 1) return lfail(EPI_EINVAL, "epi_mlp_train_step: bad argument");
    Acts a;
    epi_status s = ensure_acts(net, rows, a);
    if (s == EPI_OK) LCK(cudaMemsetAsync(net->status, 0, 4, net->stream));
    if (s == EPI_OK) s = forward(net, X_dev, rows, a, a.Y, true);
    if (s == EPI_OK) s = backward(net, t_dev, rows, a);
    if (s != EPI_OK) return s;
    net->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)net->step), c2 = 1.0f - std::pow(b2, (float)net->step);
    learn::adamw_kernel<<<blocks_for(net->n_params), 256, 0, net->stream>>>(net->w, net->g, net->m1, net->m2, net->wb,
                                                                          net->n_params, lr, b1, b2, 1e-8f, wd, c1, c2);
    LCK(cudaGetLastError());
    if (loss_host) {
        // the status word is only ever set by a tensor-core wait that gave up
        int32_t hs = 0;
        LCK(cudaMemcpyAsync(loss_host, a.loss, 4, cudaMemcpyDeviceToHost, net->stream));
        LCK(cudaMemcpyAsync(&hs, net->status, 4, cudaMemcpyDeviceToHost, net->stream));
        LCK(cudaStreamSynchronize(net->stream));
        if (hs) return lfail(EPI_ETIMEOUT, "epi_mlp_train_step: a tensor-core wait gave up");
    }
    return EPI_OK;
}

epi_status epi_heuristic5(epi_ctx *ctx, const float *X_dev, int64_t count, int n_feat, float *out_dev)
{
    if (!ctx || !X_dev || !out_dev || count < 0) return lfail(EPI_EINVAL, "epi_heuristic5: bad argument");
    if (n_feat != 25 && n_feat != 30) return lfail(EPI_EINVAL, "epi_heuristic5: n_feat must be 25 or 30");
    if (count == 0) return EPI_OK;
    cudaSetDevice(epi_ctx_device(ctx));
    learn::heuristic5_kernel<<<blocks_for(count), 256, 0, epi_ctx_stream(ctx)>>>(X_dev, count, n_feat, out_dev);
    LCK(cudaGetLastError());
    return EPI_OK;
}

}  // extern "C"

// dataset-side kernels of the proposer
namespace epi {

epi_status mlp_forward_rows(epi_mlp *net, const float *X, int64_t max_rows, const uint32_t *idx, const int32_t *n_dev,
                            float *y)
{
    if (!(net->forward_path != 1 && mlp_tc_applies(net->n_in, net->hidden))) return EPI_EUNSUPPORTED;
    if (max_rows < 1) return EPI_OK;
    const Offs o = offsets(net->n_in, net->hidden);
    LCK(cudaMemsetAsync(net->status, 0, 4, net->stream));
    LCK(launch_mlp_forward_tc(X, max_rows, idx, n_dev, net->n_in, net->norm, net->wb + o.W1, net->w + o.b1,
                              net->wb + o.W2, net->w + o.b2, net->wb + o.W3, net->w + o.b3, y, net->status,
                              net->num_sms, net->stream));
    int32_t st = 0;
    LCK(cudaMemcpyAsync(&st, net->status, 4, cudaMemcpyDeviceToHost, net->stream));
    LCK(cudaStreamSynchronize(net->stream));
    if (st) return lfail(EPI_ETIMEOUT, "network inference: a tensor-core wait gave up");
    return EPI_OK;
}

cudaError_t launch_features5(const DevData &d, const float *s1, const float *s2, const float *s3, const float *s4,
                             const uint32_t *combs, int64_t count, float *X, cudaStream_t st)
{
    learn::features5_kernel<<<blocks_for(count), 256, 0, st>>>(d, s1, s2, s3, s4, combs, count, X);
    return cudaGetLastError();
}

cudaError_t launch_candidates5(const DevData &d, const uint32_t *triples, int64_t first, int64_t count,
                               uint32_t *combs, const float *s3, uint8_t *keep, cudaStream_t st)
{
    learn::candidates5_kernel<<<blocks_for(count), 256, 0, st>>>(d, triples, first, count, combs, s3, keep);
    return cudaGetLastError();
}

cudaError_t launch_candidates5_at(const DevData &d, const uint32_t *triples, const uint64_t *idx, int64_t count,
                                  uint32_t *combs, cudaStream_t st)
{
    learn::candidates5_at_kernel<<<blocks_for(count), 256, 0, st>>>(d, triples, idx, count, combs);
    return cudaGetLastError();
}

cudaError_t launch_cand_features5(const DevData &d, const uint32_t *triples, int64_t first, int64_t count,
                                  const float *s1, const float *s2, const float *s3, const float *s4, float *X,
                                  uint8_t *keep, uint32_t *combs, cudaStream_t st)
{
    learn::cand_features5_kernel<<<blocks_for(count), 256, 0, st>>>(d, triples, first, count, s1, s2, s3, s4, X,
                                                                    keep, combs);
    return cudaGetLastError();
}

cudaError_t launch_lookup(const DevData &d, int k, const float *table, const uint32_t *combs, int64_t count,
                          float *out, cudaStream_t st)
{
    learn::lookup_kernel<<<blocks_for(count), 256, 0, st>>>(d, k, table, combs, count, out);
    return cudaGetLastError();
}


}  // namespace epi
