// Dataset construction on the device: genotype tables (Section 2.1, Fig. 2)
// and the binomial table used for lexicographic (un)ranking.
#include "epi_internal.cuh"
#include "epi_host.h"

namespace epi {

// One block: position of every individual inside its subtable (cases and
// controls each keep input order), the inverse maps, and the class sizes.
// Phenotype values outside {0, 1} set ST_BAD_PHENO.
__global__ void __launch_bounds__(1024) scan_pheno_kernel(const uint8_t *__restrict__ pheno, int64_t m,
                                                          int32_t *__restrict__ case_idx,
                                                          int32_t *__restrict__ ctrl_idx,
                                                          int64_t *__restrict__ m1_out,
                                                          int32_t *__restrict__ status)
{
    __shared__ int64_t part[1024];
    const int64_t per = (m + blockDim.x - 1) / blockDim.x;
    const int64_t b = (int64_t)threadIdx.x * per;
    const int64_t e = min(m, b + per);
    int64_t cnt = 0;
    bool bad = false;
    for (int64_t i = b; i < e; i++) {
        const uint8_t y = pheno[i];
        bad |= y > 1;
        cnt += (y == 1);
    }
    if (bad) atomicOr(status, ST_BAD_PHENO);
    part[threadIdx.x] = cnt;
    __syncthreads();
    // inclusive scan of the per-thread case counts (Hillis-Steele)
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t c = part[threadIdx.x] - cnt;          // cases before this slice
    int64_t n0 = b - c;                           // controls before this slice
    for (int64_t i = b; i < e; i++) {
        if (pheno[i] == 1) case_idx[c++] = (int32_t)i;
        else ctrl_idx[n0++] = (int32_t)i;
    }
    if (threadIdx.x == blockDim.x - 1) *m1_out = part[threadIdx.x];
}

// One warp per (SNP, 32-individual word of a subtable): lane b loads the
// genotype of individual 32 w + b and three ballots give the three rows.
// Pad bits (past the subtable's size) stay 0.  Genotypes above 2 set
// ST_BAD_GENO.  With m1_check given (the case count the scan kernel found on
// the device), a class size m1 that differs from it means the index maps hold
// fewer written entries than m1 / m0 claim: then no index is read and every
// row is written as zeros (the caller reports the mismatch).
__global__ void pack_masks_kernel(const uint8_t *__restrict__ geno, int64_t n, int64_t m,
                                  const int32_t *__restrict__ case_idx, const int32_t *__restrict__ ctrl_idx,
                                  int64_t m1, int32_t W1, int32_t Wt, uint32_t *__restrict__ masks,
                                  int32_t *__restrict__ status, const int64_t *__restrict__ m1_check)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t total = n * Wt;
    const bool counts_ok = m1_check == nullptr || *m1_check == m1;
    const int64_t m0 = counts_ok ? m - m1 : 0;
    if (!counts_ok) m1 = 0;
    for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < total; wi += warps) {
        const int64_t s = wi / Wt;
        const int32_t w = (int32_t)(wi - s * Wt);
        int64_t pos;
        const int32_t *idx;
        int64_t lim;
        if (w < W1) { pos = (int64_t)w * 32 + lane; idx = case_idx; lim = m1; }
        else { pos = (int64_t)(w - W1) * 32 + lane; idx = ctrl_idx; lim = m0; }
        int g = 3;                                // 3 = no individual
        if (pos < lim) {
            g = geno[s * m + idx[pos]];
            if (g > 2) { atomicOr(status, ST_BAD_GENO); g = 3; }
        }
        const uint32_t r0 = __ballot_sync(0xffffffffu, g == 0);
        const uint32_t r1 = __ballot_sync(0xffffffffu, g == 1);
        const uint32_t r2 = __ballot_sync(0xffffffffu, g == 2);
        if (lane < 3) {
            const uint32_t v = lane == 0 ? r0 : (lane == 1 ? r1 : r2);
            masks[(s * 3 + lane) * Wt + w] = v;
        }
    }
}

// C(a, b) for 0 <= a <= n, 0 <= b <= 8, exact or saturated to ~0.
__global__ void binom_kernel(int64_t n, uint64_t *__restrict__ tab)
{
    const int64_t total = 9 * (n + 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / (n + 1));
        const int64_t a = i - (int64_t)b * (n + 1);
        uint64_t v = 0;
        if (a >= b) {
            unsigned __int128 r = 1;
            bool sat = false;
            for (int t = 0; t < b; t++) {
                r = r * (unsigned __int128)(a - t) / (unsigned __int128)(t + 1);
                if (r > (unsigned __int128)(~0ull)) { sat = true; break; }
            }
            v = sat ? kBinomSaturated : (uint64_t)r;
        }
        tab[i] = v;
    }
}

void launch_scan_pheno(const uint8_t *pheno, int64_t m, int32_t *case_idx, int32_t *ctrl_idx, int64_t *m1,
                       int32_t *status, cudaStream_t st)
{
    scan_pheno_kernel<<<1, 1024, 0, st>>>(pheno, m, case_idx, ctrl_idx, m1, status);
}

void launch_pack_masks(const uint8_t *geno, int64_t n, int64_t m, const int32_t *case_idx, const int32_t *ctrl_idx,
                       int64_t m1, int32_t W1, int32_t Wt, uint32_t *masks, int32_t *status, int num_sms,
                       cudaStream_t st, const int64_t *m1_check)
{
    const int64_t warps = n * (int64_t)Wt;
    int64_t blocks = (warps + 7) / 8;
    const int64_t cap = (int64_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    pack_masks_kernel<<<(unsigned)blocks, 256, 0, st>>>(geno, n, m, case_idx, ctrl_idx, m1, W1, Wt, masks, status,
                                                       m1_check);
}

void launch_binom(int64_t n, uint64_t *tab, int num_sms, cudaStream_t st)
{
    int64_t blocks = (9 * (n + 1) + 255) / 256;
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    binom_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, tab);
}

}  // namespace epi
