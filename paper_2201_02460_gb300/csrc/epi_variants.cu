// Last-level counting with different instructions: the GPU counterpart of
// the paper's comparison of popcount implementations for building
// contingency tables (Section 3.1, Table 1).
//
// Every variant computes the same thing, the contingency table of every
// k-combination (Section 2.2): for each prefix (the first k-1 SNPs, in
// lexicographic order) its genotype table P[x'] = AND of the prefix SNPs'
// rows (Section 2.1, Fig. 2) is built once in shared memory, then for every
// last SNP j after the prefix
//     n_y[x' 3 + g] = sum over the words w of class y of count(P[x'][w] & M[j][g][w])
// for g = 0, 1, and genotype 2 by subtraction from the row total of P[x'].
// Only the count differs:
//   variant 0  POPC: the 32-bit population-count instruction;
//   variant 1  LUT: four lookups of a 256-entry byte table in shared memory
//              (the table-lookup popcount of CPU kernels);
//   variant 2  binary MMA: mma.sync m16n8k256 with AND + POPC on the
//              tensor cores (16 prefix rows x 4 last SNPs x 2 genotypes per
//              instruction, 256 individuals deep).
// The tensor-core FP8 0/1 GEMM (epi_tc.cu) is the fourth way and is timed by
// the search itself.  Each kernel folds every count into a checksum that
// does not depend on the order of the work, and can also write every table.
#include <cuda_runtime.h>

#include "epi_host.h"
#include "epi_internal.cuh"

namespace epi {
namespace variants {

constexpr int kThreads = 128;

template <int K>
struct Shape {
    static constexpr int R = K == 2 ? 3 : (K == 3 ? 9 : 27);   // prefix rows
};

// Words of a prefix row in shared memory: Wt + 4, so that the 8 rows and 4
// word offsets one MMA fragment load touches fall in 32 distinct banks.
__host__ __device__ inline int row_stride(int32_t Wt) { return Wt + 4; }

__host__ __device__ inline size_t smem_bytes(int R, int32_t Wt)
{
    return (size_t)R * row_stride(Wt) * 4 + (size_t)R * 2 * 4 + 256 * 4;
}

// Weight of one count in the checksum: distinct for every (cell, class) so a
// count in the wrong cell changes the sum.
__device__ __forceinline__ uint64_t cell_weight(int cells, int y, int x) { return 1 + (uint64_t)x + (uint64_t)y * cells; }

// Lexicographic rank of (prefix, j) among the k-subsets (first SNP most
// significant).
template <int K>
__device__ __forceinline__ uint64_t comb_rank(const DevData &d, uint64_t total, const int32_t *pre, int32_t j)
{
    uint64_t s = 0;
#pragma unroll
    for (int t = 0; t < K - 1; t++) s += binom_at(d.binom, d.n, d.n - 1 - pre[t], K - t);
    s += (uint64_t)(d.n - 1 - j);
    return total - 1 - s;
}

// The prefix's table rows and their per-class totals into shared memory.
template <int K>
__device__ void build_prefix(const DevData &d, const int32_t *pre, uint32_t *P, uint32_t *T)
{
    constexpr int R = Shape<K>::R;
    const int ws = row_stride(d.Wt);
    for (int i = threadIdx.x; i < R * 2; i += blockDim.x) T[i] = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < R * d.Wt; idx += blockDim.x) {
        const int x = idx / d.Wt, w = idx - x * d.Wt;
        uint32_t v = 0xffffffffu;
        int rem = x, div = R / 3;
#pragma unroll
        for (int t = 0; t < K - 1; t++) {
            const int g = rem / div;
            rem -= g * div;
            div = div > 1 ? div / 3 : 1;
            v &= d.masks[((int64_t)pre[t] * 3 + g) * d.Wt + w];
        }
        P[x * ws + w] = v;
        atomicAdd(&T[x * 2 + (w < d.W1 ? 0 : 1)], (uint32_t)__popc(v));
    }
    __syncthreads();
}

template <int V>
__device__ __forceinline__ uint32_t count_bits(uint32_t x, const uint32_t *lut)
{
    if constexpr (V == 0) return (uint32_t)__popc(x);
    else return lut[x & 255u] + lut[(x >> 8) & 255u] + lut[(x >> 16) & 255u] + lut[x >> 24];
}

// Variants 0 and 1: one thread per last SNP, its two genotype rows read once
// per word and counted against every prefix row (read from shared memory as
// a broadcast), nine rows at a time.
template <int K, int V>
__global__ void __launch_bounds__(kThreads) count_rows_kernel(DevData d, uint64_t total, uint64_t n_prefix,
                                                              uint32_t *__restrict__ tables,
                                                              unsigned long long *__restrict__ checksum)
{
    constexpr int R = Shape<K>::R;
    constexpr int G = R < 9 ? R : 9;
    constexpr int cells = R * 3;
    extern __shared__ __align__(16) uint32_t sm[];
    const int ws = row_stride(d.Wt);
    uint32_t *P = sm;
    uint32_t *T = P + R * ws;
    uint32_t *lut = T + R * 2;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = (uint32_t)__popc(i);
    __shared__ int32_t pre[K];
    uint64_t acc = 0;
    for (uint64_t q = blockIdx.x; q < n_prefix; q += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) unrank_lex(d.binom, d.n, K - 1, q, pre);
        __syncthreads();
        const int32_t c = pre[K - 2];
        if (c >= d.n - 1) continue;
        build_prefix<K>(d, pre, P, T);
        for (int32_t j = c + 1 + threadIdx.x; j < d.n; j += blockDim.x) {
            const uint32_t *m0 = d.masks + ((int64_t)j * 3 + 0) * d.Wt;
            const uint32_t *m1 = d.masks + ((int64_t)j * 3 + 1) * d.Wt;
            const uint64_t rank = tables ? comb_rank<K>(d, total, pre, j) : 0;
#pragma unroll 1
            for (int x0 = 0; x0 < R; x0 += G) {
#pragma unroll 1
                for (int y = 0; y < 2; y++) {
                    uint32_t a[G], b[G];
#pragma unroll
                    for (int r = 0; r < G; r++) { a[r] = 0; b[r] = 0; }
                    const int w0 = y ? d.W1 : 0, w1 = y ? d.Wt : d.W1;
                    for (int w = w0; w < w1; w++) {
                        const uint32_t g0 = __ldg(m0 + w), g1 = __ldg(m1 + w);
#pragma unroll
                        for (int r = 0; r < G; r++) {
                            const uint32_t p = P[(x0 + r) * ws + w];
                            a[r] += count_bits<V>(p & g0, lut);
                            b[r] += count_bits<V>(p & g1, lut);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < G; r++) {
                        const int x = x0 + r;
                        const uint32_t n2 = T[x * 2 + y] - a[r] - b[r];
                        acc += a[r] * cell_weight(cells, y, 3 * x) + b[r] * cell_weight(cells, y, 3 * x + 1) +
                               n2 * cell_weight(cells, y, 3 * x + 2);
                        if (tables) {
                            uint32_t *o = tables + rank * 2 * cells + (size_t)y * cells + 3 * x;
                            o[0] = a[r]; o[1] = b[r]; o[2] = n2;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(checksum, (unsigned long long)acc);
}

// One m16n8k256 binary MMA with AND + POPC: C[16 x 8] += popc(A[16 x 256] &
// B[256 x 8]) over 32-bit words of k.  Fragments (per lane, g = lane / 4,
// t = lane % 4): a0 = A[g][word t], a1 = A[g + 8][word t], a2 = A[g][word
// t + 4], a3 = A[g + 8][word t + 4]; b0 = B[word t][col g], b1 = B[word
// t + 4][col g]; c0, c1 = C[g][2t, 2t + 1], c2, c3 = C[g + 8][2t, 2t + 1].
__device__ __forceinline__ void mma_b1_and_popc(uint32_t (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Variant 2: each warp takes 4 last SNPs at a time (8 B columns: SNP
// j0 + g' / 2, genotype g' % 2) against all prefix rows (M tiles of 16),
// separately over the case words and the control words (8 words = 256
// individuals per instruction; words past the class end enter as zeros).
template <int K>
__global__ void __launch_bounds__(kThreads) count_mma_kernel(DevData d, uint64_t total, uint64_t n_prefix,
                                                             uint32_t *__restrict__ tables,
                                                             unsigned long long *__restrict__ checksum)
{
    constexpr int R = Shape<K>::R;
    constexpr int MT = (R + 15) / 16;
    constexpr int cells = R * 3;
    extern __shared__ __align__(16) uint32_t sm[];
    const int ws = row_stride(d.Wt);
    uint32_t *P = sm;
    uint32_t *T = P + R * ws;
    __shared__ int32_t pre[K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint64_t acc = 0;
    for (uint64_t q = blockIdx.x; q < n_prefix; q += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) unrank_lex(d.binom, d.n, K - 1, q, pre);
        __syncthreads();
        const int32_t c = pre[K - 2];
        if (c >= d.n - 1) continue;
        build_prefix<K>(d, pre, P, T);
        for (int32_t j0 = c + 1 + 4 * warp; j0 < d.n; j0 += 4 * (kThreads / 32)) {
            // this lane's B column: SNP jb, genotype gb
            const int32_t jb = j0 + (g >> 1);
            const int gb = g & 1;
            const uint32_t *mrow = d.masks + ((int64_t)(jb < d.n ? jb : 0) * 3 + gb) * d.Wt;
#pragma unroll 1
            for (int y = 0; y < 2; y++) {
                const int w0 = y ? d.W1 : 0, w1 = y ? d.Wt : d.W1;
                uint32_t cacc[MT][4];
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
#pragma unroll
                    for (int e = 0; e < 4; e++) cacc[mt][e] = 0;
                for (int kb = w0; kb < w1; kb += 8) {
                    const int wa = kb + t, wb = kb + t + 4;
                    const uint32_t b0 = (jb < d.n && wa < w1) ? __ldg(mrow + wa) : 0u;
                    const uint32_t b1 = (jb < d.n && wb < w1) ? __ldg(mrow + wb) : 0u;
#pragma unroll
                    for (int mt = 0; mt < MT; mt++) {
                        const int r0 = mt * 16 + g, r1 = r0 + 8;
                        uint32_t a[4];
                        a[0] = (r0 < R && wa < w1) ? P[r0 * ws + wa] : 0u;
                        a[1] = (r1 < R && wa < w1) ? P[r1 * ws + wa] : 0u;
                        a[2] = (r0 < R && wb < w1) ? P[r0 * ws + wb] : 0u;
                        a[3] = (r1 < R && wb < w1) ? P[r1 * ws + wb] : 0u;
                        mma_b1_and_popc(cacc[mt], a, b0, b1);
                    }
                }
                // C[row][col]: col 2t + e is SNP j0 + t, genotype e
                const int32_t j = j0 + t;
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int x = mt * 16 + g + 8 * h;
                        if (x >= R || j >= d.n) continue;
                        const uint32_t n0 = cacc[mt][2 * h], n1 = cacc[mt][2 * h + 1];
                        const uint32_t n2 = T[x * 2 + y] - n0 - n1;
                        acc += n0 * cell_weight(cells, y, 3 * x) + n1 * cell_weight(cells, y, 3 * x + 1) +
                               n2 * cell_weight(cells, y, 3 * x + 2);
                        if (tables) {
                            uint32_t *o = tables + comb_rank<K>(d, total, pre, j) * 2 * cells + (size_t)y * cells + 3 * x;
                            o[0] = n0; o[1] = n1; o[2] = n2;
                        }
                    }
            }
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) atomicAdd(checksum, (unsigned long long)acc);
}

}  // namespace variants

size_t count_variant_smem_bytes(int k, int32_t Wt)
{
    const int R = k == 2 ? 3 : (k == 3 ? 9 : 27);
    return variants::smem_bytes(R, Wt);
}

// Counts every table of order k (2..4) with the chosen variant; `tables`
// (device, [C(n,k)][2][3^k]) may be NULL.
cudaError_t launch_count_variant(const DevData &d, int k, int variant, uint64_t total, uint32_t *tables,
                                 unsigned long long *checksum, int grid, cudaStream_t st)
{
    const size_t smem = count_variant_smem_bytes(k, d.Wt);
    const uint64_t n_prefix = host_binom(d.n, k - 1);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, variants::kThreads, smem, st>>>(d, total, n_prefix, tables, checksum);
        return cudaGetLastError();
    };
    if (variant == 0)
        return k == 2 ? run(variants::count_rows_kernel<2, 0>) : k == 3 ? run(variants::count_rows_kernel<3, 0>)
                                                                        : run(variants::count_rows_kernel<4, 0>);
    if (variant == 1)
        return k == 2 ? run(variants::count_rows_kernel<2, 1>) : k == 3 ? run(variants::count_rows_kernel<3, 1>)
                                                                        : run(variants::count_rows_kernel<4, 1>);
    return k == 2 ? run(variants::count_mma_kernel<2>) : k == 3 ? run(variants::count_mma_kernel<3>)
                                                                : run(variants::count_mma_kernel<4>);
}

}  // namespace epi
