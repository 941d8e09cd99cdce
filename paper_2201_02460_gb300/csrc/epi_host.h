// Host-side launchers of libepi's kernels (one definition per .cu file).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "epi_internal.cuh"

namespace epi {

// exact C(n, k), or UINT64_MAX when it does not fit
inline uint64_t host_binom(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 r = 1;
    for (int64_t i = 0; i < k; i++) {
        r = r * (unsigned __int128)(n - i) / (unsigned __int128)(i + 1);
        if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
    }
    return (uint64_t)r;
}

// epi_data.cu
void launch_scan_pheno(const uint8_t *pheno, int64_t m, int32_t *case_idx, int32_t *ctrl_idx, int64_t *m1,
                       int32_t *status, cudaStream_t st);
// m1_check (device, may be NULL): the case count found by scan_pheno; where it
// differs from m1 the index maps are not read and the rows are zeros
void launch_pack_masks(const uint8_t *geno, int64_t n, int64_t m, const int32_t *case_idx, const int32_t *ctrl_idx,
                       int64_t m1, int32_t W1, int32_t Wt, uint32_t *masks, int32_t *status, int num_sms,
                       cudaStream_t st, const int64_t *m1_check = nullptr);
void launch_binom(int64_t n, uint64_t *tab, int num_sms, cudaStream_t st);

// epi_popc.cu
bool popc_row_group_ok(int k, int R);
bool popc_global_prefix_ok(int k, int R);
int popc_default_row_group(int k);
int popc_slot_words(int k, int32_t Wt);
// shared memory of one CTA; with global_prefix the prefix tables live in a
// global buffer of grid x slots x popc_slot_words words instead
size_t popc_smem_bytes(int k, int32_t Wt, int slots, int cand_p2, bool global_prefix = false);
int popc_max_active(int k, int R, size_t smem, bool global_prefix = false);
cudaError_t launch_popc_search(const DevData &d, int k, int R, uint64_t rank_begin, uint64_t rank_end, int tile,
                               int pool, int slots, int cand_p2, uint32_t *global_thr, float *list_score,
                               uint64_t *list_rank, int32_t *list_count, int grid, size_t smem, cudaStream_t st,
                               float *all_scores = nullptr, uint32_t *pre_global = nullptr,
                               uint32_t *pair_sing = nullptr, int top_n = 0);
// orders 6-8: whether a search runs the (k-2)-prefix kernel, and the words of
// one CTA's single-count table for it (pair_sing above: grid x that many)
bool popc_pair_applies(int k, int32_t Wt, int pool, bool all_scores);
int64_t popc_pair_sing_words(int k, int64_t n);
int popc_pair_grid(int num_sms, int k, int64_t n);
// batched: one launch over several datasets of order k (descriptors in device memory)
size_t popc_ds_bytes();
void popc_fill_ds(void *dst, const DevData &d, uint64_t rank_begin, uint64_t rank_end, int cta_begin, int cta_count,
                  uint32_t *global_thr);
cudaError_t launch_popc_batch(const void *ds_dev, const int32_t *cta_ds_dev, int k, int R, int max_wt, int tile,
                              int pool, int slots, int cand_p2, float *list_score, uint64_t *list_rank,
                              int32_t *list_count, int grid, size_t smem, cudaStream_t st);

// epi_tc.cu
size_t tc_b8_bytes(const DevData &d);
// comb_p: 0 = E4M3 operand of the separate-class variant, else the E5M2
// operand of the combined-class variant with class shift comb_p
cudaError_t launch_build_b8(const DevData &d, unsigned char *b8, int num_sms, cudaStream_t st, int comb_p);
// class shift of the combined-class variant for an order-k search, 0 where
// the separate-class variant runs
int tc_comb_shift(const DevData &d, int k);
// work items of the whole search (separate-class tiles), or of the prefixes
// with first SNP in [a, b] for N tiles of kj last SNPs
uint64_t tc_item_count(int64_t n, int k);
uint64_t tc_item_count(int64_t n, int k, int64_t a, int64_t b, int kj);
// first SNP of the combination of lexicographic rank r
int64_t tc_first_snp(int64_t n, int k, uint64_t r);
// combinations the tensor path counts to search the rank range [rb, re)
uint64_t tc_range_work(int64_t n, int k, uint64_t rb, uint64_t re);
// entries of a CTA's candidate buffer for a pool; shared memory of one CTA
// with that buffer in shared memory or (cand_global) in a global buffer
int tc_cand_p2(int k, int pool, bool comb = false);
size_t tc_smem_bytes(int cand_p2, int k, bool cand_global, bool comb = false);
// item_cum: device [2][n + 1] (item and prefix tables); ranks [rb, re);
// cand_g / rank_g: NULL, or [grid][tc_cand_p2] global candidate buffers;
// comb_p: 0 = separate-class variant (b8 built with comb_p 0), else the
// combined-class variant (b8 built with the same comb_p)
cudaError_t launch_tc_search(const DevData &d, int k, const unsigned char *b8, uint64_t *item_cum, int pool,
                             uint32_t *global_thr, float *list_score, uint64_t *list_rank, int32_t *list_count,
                             int32_t *status, int grid, uint64_t total, uint64_t rb, uint64_t re, cudaStream_t st,
                             int *cand_p2_out, float *cand_g, uint64_t *rank_g, uint32_t *dump = nullptr,
                             unsigned long long *waits = nullptr, unsigned long long wait_ns = 0, int comb_p = 0);
constexpr int kTcWaitSlots = 8;
// batched tensor-core launches: per-dataset descriptors and B-operand maps
// (128-byte CUtensorMap, 64-byte aligned) live in device memory
size_t tc_ds_bytes();
cudaError_t launch_tc_item_cum(const DevData &d, int k, uint64_t rb, uint64_t re, uint64_t *item_cum,
                               cudaStream_t st, bool comb = false);
cudaError_t tc_fill_batch_entry(void *ds_host, void *tmap_host, const DevData &d, int k, const unsigned char *b8,
                                uint64_t *item_cum, uint32_t *global_thr, uint64_t total, const void *tmap_dev,
                                int cta_begin, int cta_count);
cudaError_t launch_tc_batch(const void *ds_dev, const int32_t *cta_ds_dev, int k, int pool, float *list_score,
                            uint64_t *list_rank, int32_t *list_count, int32_t *status, int grid, cudaStream_t st,
                            float *cand_g, uint64_t *rank_g);

// epi_peak.cu: tensor-pipe rate of the counting MMA (one CTA per SM,
// `stages` groups of four M128 N128 K32 FP8 MMAs; per-CTA cycles)
size_t mma_rate_smem_bytes(int shape);
cudaError_t launch_mma_rate(int shape, int64_t stages, unsigned long long *cycles, int32_t *status, int grid,
                            cudaStream_t st);

// epi_variants.cu: every table of order k (2..4) counted with the POPC
// instruction (variant 0), a byte lookup table (1) or binary MMA (2)
size_t count_variant_smem_bytes(int k, int32_t Wt);
cudaError_t launch_count_variant(const DevData &d, int k, int variant, uint64_t total, uint32_t *tables,
                                 unsigned long long *checksum, int grid, cudaStream_t st);

// epi_gemm_tc.cu: C = A . B^T on tcgen05 (BF16 K-major operands, FP32 C),
// K split over CTAs into `partial` (gemm_tc_partial_floats floats, or NULL)
size_t gemm_tc_smem_bytes(int nt);
size_t gemm_tc_partial_floats(int M, int N, int K, int num_sms);
cudaError_t launch_gemm_tc(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc, int M, int N,
                           int K, float *partial, int32_t *status, int num_sms, cudaStream_t st);

// epi_learn.cu (proposer)
cudaError_t launch_features5(const DevData &d, const float *s1, const float *s2, const float *s3, const float *s4,
                             const uint32_t *combs, int64_t count, float *X, cudaStream_t st);
cudaError_t launch_candidates5(const DevData &d, const uint32_t *triples, int64_t first, int64_t count,
                               uint32_t *combs, const float *s3, uint8_t *keep, cudaStream_t st);
cudaError_t launch_candidates5_at(const DevData &d, const uint32_t *triples, const uint64_t *idx, int64_t count,
                                  uint32_t *combs, cudaStream_t st);
// epi_mlp_tc.cu
size_t mlp_tc_smem_bytes();
bool mlp_tc_applies(int n_in, int hidden);
cudaError_t launch_mlp_forward_tc(const float *X, int64_t rows, const uint32_t *idx, const int32_t *rows_dev, int n_in,
                                  const float *norm, const void *W1, const float *b1, const void *W2, const float *b2,
                                  const void *W3, const float *b3, float *y, int32_t *status, int num_sms,
                                  cudaStream_t st);
// Tensor-core predictions for the listed rows only: row j < *n_dev (at most
// max_rows) is X[idx[j]], its prediction goes to y[idx[j]]; waits for the
// kernel.  EPI_EUNSUPPORTED where the fused kernel does not apply.
epi_status mlp_forward_rows(epi_mlp *net, const float *X, int64_t max_rows, const uint32_t *idx, const int32_t *n_dev,
                            float *y);
cudaError_t launch_cand_features5(const DevData &d, const uint32_t *triples, int64_t first, int64_t count,
                                  const float *s1, const float *s2, const float *s3, const float *s4, float *X,
                                  uint8_t *keep, uint32_t *combs, cudaStream_t st);
cudaError_t launch_lookup(const DevData &d, int k, const float *table, const uint32_t *combs, int64_t count,
                          float *out, cudaStream_t st);
// epi_topk.cu: the k best of count scores (score desc, index asc; keep may
// be NULL), by radix select; sorted (k <= 4096) or as an unordered set;
// scratch of topk_scratch_bytes(k) device bytes
size_t topk_scratch_bytes(int64_t k);
cudaError_t launch_topk(const float *scores, const uint8_t *keep, int64_t count, int64_t k, void *scratch, bool sorted,
                        float *out_s, uint64_t *out_i, int32_t *out_n, int num_sms, cudaStream_t st);

// epi_select.cu
// floor: below every score to merge (the search's scores are >= 0)
cudaError_t launch_merge(const float *ls, const uint64_t *lr, const int32_t *lc, int nlists, int stride, int pool,
                         float *out_s, uint64_t *out_r, int32_t *out_n, cudaStream_t st, float floor = -1.0f);
cudaError_t launch_rescore(const DevData &d, int k, int pool, const uint64_t *cand_r, const int32_t *cand_n,
                           uint32_t *counts, double *mi64, int32_t *combs, cudaStream_t st);
cudaError_t launch_finalize(const DevData &d, int k, int top_n, int pool, const float *cand_s, const uint64_t *cand_r,
                            const int32_t *cand_n, const double *mi64, const int32_t *combs, const uint32_t *counts,
                            const uint32_t *global_thr, uint64_t total, epi_result *out, uint32_t *out_counts,
                            int32_t *n_out, int32_t *status, cudaStream_t st);
cudaError_t launch_tables(const DevData &d, int k, const uint32_t *combs, int64_t count, uint32_t *out, int num_sms,
                          cudaStream_t st);
// ranks of the scores >= thr (unordered; at most cap written, *n counts all)
cudaError_t launch_select_ge(const float *scores, int64_t count, float thr, uint64_t rank_base, uint64_t *out,
                             uint64_t cap, unsigned long long *n, int num_sms, cudaStream_t st);
cudaError_t launch_unrank(const DevData &d, int k, const uint64_t *ranks, int64_t count, uint32_t *combs,
                          cudaStream_t st);
cudaError_t launch_publish_status(const int32_t *bits, int32_t *code, cudaStream_t st);
cudaError_t launch_score_tables(const DevData &d, int k, const uint32_t *tabs, int64_t count, float *f32, double *f64,
                                int num_sms, cudaStream_t st);
// exact FP32 MI of order-5 sets [count][5] (tables counted in registers, not
// stored)
cudaError_t launch_score5_f32(const DevData &d, const uint32_t *combs, int64_t count, float *out, int num_sms,
                              cudaStream_t st);

}  // namespace epi

// context accessors for the other translation units (epi_api.cu)
struct epi_ctx;
struct epi_dataset;
cudaStream_t epi_ctx_stream(const epi_ctx *ctx);
int epi_ctx_device(const epi_ctx *ctx);
int epi_ctx_num_sms(const epi_ctx *ctx);
void epi_ctx_count_launches(epi_ctx *ctx, int n);
epi_ctx *epi_dataset_ctx(const epi_dataset *ds);
epi::DevData epi_dataset_dev(const epi_dataset *ds);
epi_status epi_dataset_lower_scores(epi_dataset *ds, int k, const float **out);
