/*
 * libepi -- exhaustive k-SNP epistasis search on one GB300 GPU (sm_103a).
 *
 * The method is that of Ponte-Fernandez et al., "A SIMD algorithm for the
 * detection of epistatic interactions of any order" (arXiv 2201.02460):
 * for every k-subset S of SNPs, build the 3^k x 2 genotype/phenotype
 * contingency table from bit-packed genotype tables (Section 2.1, Fig. 2),
 * the last combination level fused with the population count (Section 2.2),
 * score it by mutual information (Section 2.3, Eq. 1-3) and keep the best N
 * (Section 2.4, Algorithm 1).
 *
 * Conventions shared by every call:
 *   - Genotypes are uint8 in {0, 1, 2} (row g of a genotype table marks
 *     genotype g), stored [n_snps][n_samples] row-major.  Phenotypes are uint8
 *     in {0 = control, 1 = case}.  Missing genotypes are not supported.
 *   - A combination is a strictly increasing tuple s_1 < ... < s_k of SNP
 *     indices.  Its cell x = sum_t g_t 3^(k-t) (first SNP most significant,
 *     the row order of a combined genotype table, Section 2.1).
 *   - Tables are uint32 [2][3^k]: index 0 = cases, 1 = controls.
 *   - MI is in nats with probabilities count / m over all m individuals and
 *     0 log 0 = 0 (Eq. 1-3).  mi_f32 is the single-precision screening score;
 *     mi is the double-precision re-score of the same table.
 *   - Results are ordered by mi descending, equal mi broken by the
 *     lexicographically smaller tuple.  n_out = min(top_n, C(n, k)).
 *   - Host pointers are read or written during the call only; the caller
 *     owns every buffer it passes.  Device pointers must be memory of the
 *     context's device.
 *   - Every call runs on the stream given to epi_create and returns after the
 *     stream has finished the call's work, unless its name ends in _async.
 *   - Errors: a call returns a status != EPI_OK, writes no output it has not
 *     documented as partially written, and leaves a message for
 *     epi_last_error() (per thread).  Device-side failures (a watchdog that
 *     expired, a candidate pool that was too small) come back as status codes;
 *     no kernel of the library traps.
 */
#ifndef EPI_H
#define EPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EPI_OK = 0,
    EPI_EINVAL = 1,        /* bad argument (value, size, pointer, order) */
    EPI_ENOMEM = 2,        /* device or host allocation failed */
    EPI_ECUDA = 3,         /* a CUDA runtime call failed */
    EPI_EUNSUPPORTED = 4,  /* valid request the library cannot run */
    EPI_ETIMEOUT = 5,      /* a bounded device wait gave up */
    EPI_EOVERFLOW = 6      /* exact top-N not guaranteed even after retries */
} epi_status;

/* Counting path of the search. */
typedef enum {
    EPI_PATH_AUTO = 0,     /* fastest exact path for the order and sizes */
    EPI_PATH_POPC = 1,     /* bitwise AND + POPC on the integer pipe */
    EPI_PATH_TC = 2        /* exact 0/1 GEMM on tcgen05 tensor cores: orders
                              2..5 with cases and controls present
                              (EPI_EUNSUPPORTED else) */
} epi_path;

/* Tensor-core counting variant (epi_set_tc_variant). */
typedef enum {
    EPI_TC_AUTO = 0,       /* order 3 with m1 * 2^p + m0 < 2^23 (2^p the
                              least power of two above m0, p <= 14): both
                              classes in one accumulator, 256-column tiles;
                              else separate case and control accumulators */
    EPI_TC_SEPARATE = 1    /* always separate case and control accumulators */
} epi_tc_variant;

#define EPI_MAX_ORDER 8    /* highest order the API accepts (Table 2 goes to 8) */

typedef struct epi_ctx epi_ctx;
typedef struct epi_dataset epi_dataset;

/* One retained combination. */
typedef struct {
    uint32_t snp[EPI_MAX_ORDER];  /* s_1 < ... < s_k; entries k.. are 0 */
    double mi;                    /* double-precision MI (nats) */
    float mi_f32;                 /* single-precision screening MI (nats) */
    uint32_t order;               /* k */
    uint64_t rank;                /* lexicographic rank among the k-subsets */
} epi_result;

/* Message of the last failed call on this thread ("" if none). */
const char *epi_last_error(void);

/* Context on CUDA device `device`; all work is queued on `cuda_stream` (a
 * cudaStream_t, NULL = the legacy default stream).  The context owns its
 * device scratch memory, allocated on first use and grown as needed.
 * epi_destroy may be called while datasets of the context are alive: the
 * context is then freed by the last epi_dataset_destroy, and no other call
 * may use it meanwhile. */
epi_status epi_create(int device, void *cuda_stream, epi_ctx **out);
void epi_destroy(epi_ctx *ctx);

/* Genotype tables of a dataset (Section 2.1).  geno [n_snps][n_samples] and
 * pheno [n_samples] are host memory when inputs_on_device = 0, device memory
 * otherwise; they are read during the call only.  The library packs them on
 * the device into per-SNP case and control bit rows.  Fails with EPI_EINVAL
 * for n_snps < 1, n_samples < 1, n_samples > 2^23 - 1 or a value outside
 * {0,1,2} / {0,1} (checked on the device for device inputs).  Device inputs
 * that are not device memory of the context's device fail with EPI_EINVAL. */
epi_status epi_dataset_create(epi_ctx *ctx, const uint8_t *geno, const uint8_t *pheno,
                              int64_t n_snps, int64_t n_samples, int inputs_on_device,
                              epi_dataset **out);
void epi_dataset_destroy(epi_dataset *ds);

/* Sizes of a dataset: n_snps, n_samples, n_cases, n_controls. */
epi_status epi_dataset_info(const epi_dataset *ds, int64_t *n_snps, int64_t *n_samples,
                            int64_t *n_cases, int64_t *n_controls);

/* Exhaustive search of every k-subset (Algorithm 1), keeping the best top_n
 * (Section 2.4).  out: host array of top_n records; counts (optional, may be
 * NULL): host array [top_n][2][3^k]; *n_out receives min(top_n, C(n,k)).
 * Orders 1..8 run on the GPU (the tensor-core path covers orders 2..5, the
 * popcount path 1..8); top_n in [1, 1024]. */
epi_status epi_search(epi_dataset *ds, int order, int top_n, int path, epi_result *out,
                      uint32_t *counts, int *n_out);

/* The same restricted to combinations of lexicographic rank in
 * [rank_begin, rank_end) (rank_end clipped to C(n,k)): the resumable and
 * shardable form of the search.  Both counting paths take ranges; the
 * tensor-core path counts every combination whose first SNP lies between
 * those of ranks rank_begin and rank_end - 1 and keeps only the range's, so
 * EPI_PATH_AUTO takes it for a range only when that adds at most the range's
 * own size of work. */
epi_status epi_search_range(epi_dataset *ds, int order, int top_n, int path,
                            uint64_t rank_begin, uint64_t rank_end, epi_result *out,
                            uint32_t *counts, int *n_out);

/* Device-side form of epi_search: results are written to device memory
 * (out_dev [top_n] records, counts_dev [top_n][2][3^k] or NULL, n_out_dev one
 * int32) and status_dev (one int32, device) receives EPI_OK or the device
 * status of the search.  Returns after queueing the work; the host does not
 * wait.  A search that needs a larger candidate pool reports EPI_EOVERFLOW in
 * status_dev instead of retrying. */
epi_status epi_search_async(epi_dataset *ds, int order, int top_n, int path,
                            epi_result *out_dev, uint32_t *counts_dev, int32_t *n_out_dev,
                            int32_t *status_dev);

/* Many independent searches at once (one per dataset, Algorithm 1 each):
 * datasets of the same order and counting path share one persistent launch
 * whose CTAs are split among them in proportion to their work, and the whole
 * batch (counting launches, per-dataset merge, re-score and selection, and
 * the copies back) is captured once into a CUDA graph that later calls with
 * the same datasets, orders and top_n replay.  ds[i] must belong to ctx;
 * orders[i] in 1..8 (at orders 6..8 one prefix table of the largest dataset
 * must fit in shared memory, else EPI_EUNSUPPORTED), top_ns[i] in 1..1024;
 * outs[i] host arrays of top_ns[i]
 * records; counts NULL or counts[i] NULL or a host array [top_ns[i]][2][3^k];
 * n_outs[i] receives the record count.  Same results as epi_search on each
 * dataset.  Destroying a dataset invalidates the cached graph. */
epi_status epi_search_batched(epi_ctx *ctx, epi_dataset *const *ds, const int *orders, const int *top_ns,
                              int n_ds, int path, epi_result *const *outs, uint32_t *const *counts,
                              int *n_outs);

/* Autotuner (the paper has no counterpart; it tunes the library's launch
 * shapes).  Times every popcount-path shape (row group of prefix rows per
 * thread, sub-tile of combinations, prefixes staged per sub-tile) on a
 * bounded rank range of this dataset and, where the tensor-core path applies,
 * the two paths; the fastest is kept in the context for every later search
 * (EPI_PATH_AUTO, batched or not) of the same order and size bucket (SNPs and
 * sample words rounded down to powers of two).  out (may be NULL) receives
 * four ints: row group, sub-tile, staged prefixes, chosen path. */
epi_status epi_autotune(epi_dataset *ds, int order, int *out);

/* The context's autotuner choices to / from a text file. */
epi_status epi_tune_save(const epi_ctx *ctx, const char *path);
epi_status epi_tune_load(epi_ctx *ctx, const char *path);

/* Contingency tables (Section 2.2) of `count` given combinations.  combs:
 * host [count][order] uint32, each strictly increasing and < n_snps;
 * out: host [count][2][3^order].  order in 1..8. */
epi_status epi_tables(epi_dataset *ds, int order, const uint32_t *combs, int64_t count,
                      uint32_t *out);

/* Single-precision and double-precision MI of `count` host tables
 * [count][2][3^order] with the dataset's class sizes (Eq. 1-3); either
 * output may be NULL. */
epi_status epi_score_tables(epi_dataset *ds, int order, const uint32_t *tables, int64_t count,
                            float *mi_f32, double *mi_f64);

/* Number of kernels the library launched on this context since creation
 * (a diagnostic counter). */
uint64_t epi_kernel_launches(const epi_ctx *ctx);

/* Validation aid: the contingency table of every combination as the
 * tensor-core counting path computes it, before any screening.  out: host
 * [C(n,k)][2][3^order] in lexicographic rank order (at most 2 GiB).  Fails
 * with EPI_EUNSUPPORTED where the tensor-core path does not apply (see
 * epi_search).  The paper has no counterpart; the tables equal those of
 * epi_tables (Section 2.2) when the path is exact. */
epi_status epi_debug_counts(epi_dataset *ds, int order, uint32_t *out);

/* Allocation-free search, for callers that cannot allocate device memory
 * (for example a plug-in inside a host framework that owns all device
 * allocations, or code with a fixed memory budget).  The paper has no
 * counterpart: this is the popcount-path search of epi_search with every
 * intermediate buffer (genotype tables, candidate lists, recount tables) in
 * one 64 MiB array that the library holds in device memory for the life of
 * the process, on every GPU that loads it.  The call performs no cudaMalloc,
 * cudaFree or other allocating call.
 *
 * Inputs, all device memory of the current device: geno [n_snps][n_samples]
 * uint8 in {0,1,2}, pheno [n_samples] uint8 in {0,1}; n_cases must equal the
 * number of ones in pheno.  Outputs, device memory: out_dev [top_n] records,
 * counts_dev [top_n][2][3^order] (may be NULL), n_out_dev one int32,
 * status_dev one int32 that receives EPI_OK, EPI_EINVAL (invalid genotype or
 * phenotype values, or n_cases that does not match), or EPI_EOVERFLOW (the
 * candidate pool could not prove the exact top N; epi_search retries in that
 * case, this call does not).  Work is queued on cuda_stream and the call
 * returns without waiting.  order in 1..5, top_n in 1..1024.  A dataset whose
 * buffers exceed the 64 MiB array fails with EPI_EINVAL before any work is
 * queued (the genotype tables take about n_snps * 3 * 2 * ceil(n_samples/128)
 * * 16 bytes).
 *
 * With invalid genotype or phenotype values or a wrong n_cases, *n_out_dev
 * is 0 and no genotype is read outside geno_dev.
 *
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) and the device's SM count and shared-memory limit,
 * and keeps them for every later call; make that first call before any stream
 * capture.  The address belongs to the runtime's primary context of the
 * device: calls made under another context of the same device, or after a
 * cudaDeviceReset in the same process, are not supported.
 * Every call uses the same array and leaves its contents behind; calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it and
 * must be serialised by the caller. */
epi_status epi_search_static(const uint8_t *geno_dev, const uint8_t *pheno_dev, int64_t n_snps,
                             int64_t n_samples, int64_t n_cases, int order, int top_n,
                             epi_result *out_dev, uint32_t *counts_dev, int32_t *n_out_dev,
                             int32_t *status_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Learned proposer for orders where the exhaustive search is out of reach.
 * The paper has no counterpart (it searches exhaustively); these calls rank
 * candidate 5-sets by a small network fed with lower-order scores, and the
 * ranked candidates are then scored exactly with epi_tables and
 * epi_score_tables.
 * ------------------------------------------------------------------------ */

/* Thresholded output (the "significant association" branch of Fig. 1, in
 * place of a top-N): every combination of `order` (1..8) whose double-
 * precision MI (Eq. 1-3) is at least `threshold`, sorted by (MI desc, rank
 * asc).  Every combination is scored in single precision by the popcount
 * path (Section 2.2 counts, in passes of `chunk` ranks, 0 = 2^28, each pass
 * holding 4 bytes per rank of device memory); those at or above
 * threshold (1 - 2 b), b the FP32 bound of the exact top-N, are recounted and
 * scored in double precision, which decides.  *n_found receives how many
 * qualify; the best min(n_found, capacity) are written to host out [capacity]
 * and, if counts is not NULL, their tables to host counts
 * [capacity][2][3^order].  Synchronous on the context's stream. */
epi_status epi_search_threshold(epi_dataset *ds, int order, double threshold, int64_t chunk, epi_result *out,
                                int64_t capacity, uint32_t *counts, int64_t *n_found);

/* Every combination's single-precision MI (Eq. 1-3), by lexicographic rank:
 * out_dev is device memory of C(n_snps, order) floats.  Orders 1..8. */
epi_status epi_score_all(epi_dataset *ds, int order, float *out_dev);

/* Combinations of `count` lexicographic ranks (device [count] uint64, each
 * below C(n_snps, order)) into device combs [count][order]. */
epi_status epi_unrank(epi_dataset *ds, int order, const uint64_t *ranks, int64_t count, uint32_t *combs);

/* The proposer features of `count` 5-sets: ln(MI + 1e-7) of the 5 SNPs,
 * the 10 pairs and the 10 triples of each set (25 features), and, when s4 is
 * given, of its 5 four-SNP subsets (30 features); each group sorted
 * descending.  s1/s2/s3/s4: device score tables of orders 1..4 from
 * epi_score_all (s4 may be NULL); combs: device [count][5] strictly
 * increasing SNP indices; X: device [count][25 or 30] floats.  Queued on the
 * context's stream. */
epi_status epi_features5(epi_dataset *ds, const float *s1, const float *s2, const float *s3, const float *s4,
                         const uint32_t *combs, int64_t count, float *X);

/* Candidate 5-sets made of one of n_triples triples (device [n_triples][3],
 * strictly increasing) and any two other SNPs: candidate index
 * t * C(n-3, 2) + r is triple t with the r-th pair (lexicographic) of the
 * remaining SNPs; writes candidates [first, first + count) to combs (device
 * [count][5], sorted).  With s3 (the order-3 table of epi_score_all) and keep
 * (device [count] bytes) both given, keep[i] = 1 exactly when candidate i's
 * triple is the best of the set's ten triples by (score desc, rank asc), so
 * that a set holding several listed triples is kept once; both NULL skips
 * this.  Queued on the context's stream. */
epi_status epi_candidates5(epi_dataset *ds, const uint32_t *triples, int64_t n_triples, int64_t first,
                           int64_t count, uint32_t *combs, const float *s3, uint8_t *keep);

/* Exact single-precision MI (Eq. 1-3 of the Section 2.2 table) of `count`
 * order-5 sets: combs device [count][5] (strictly increasing SNP indices
 * below n_snps), out device [count] floats.  The tables are counted in
 * registers and not stored (one warp per set); the value agrees with the
 * FP32 score of epi_score_tables within the same error bound (the cell terms
 * are summed in another order).  Queued on the context's stream. */
epi_status epi_score5(epi_dataset *ds, const uint32_t *combs, int64_t count, float *out);

/* out[i] = table[lexicographic rank of combs[i]] for an order-`order` table
 * of epi_score_all (device arrays; combs [count][order] strictly increasing). */
epi_status epi_lookup(epi_dataset *ds, int order, const float *table, const uint32_t *combs, int64_t count,
                      float *out);

/* The k largest of `count` device floats (ties: smaller index first),
 * skipping entries whose keep byte is 0 when keep (device [count]) is given:
 * device outputs out_scores [k], out_index [k], n_out one int32.  k in
 * 1..4096.  NaN scores are never selected. */
epi_status epi_topk(epi_ctx *ctx, const float *scores, const uint8_t *keep, int64_t count, int k, float *out_scores,
                    uint64_t *out_index, int32_t *n_out);

/* The ranking without a network, for comparison: for rows of n_feat = 25
 * features (device X [count][25]) the sum of the ten three-way features, for
 * n_feat = 30 the sum of the five four-way features; into device out. */
epi_status epi_heuristic5(epi_ctx *ctx, const float *X_dev, int64_t count, int n_feat, float *out_dev);

/* A multilayer perceptron n_in -> hidden -> hidden -> 1 with ReLU, BF16
 * weights and activations, FP32 accumulation and FP32 master weights for the
 * optimiser; parameters in the order W1 [hidden][n_in], b1, W2
 * [hidden][hidden], b2, W3 [hidden], b3.  He-uniform initialisation from
 * `seed`.  Work runs on the context's stream. */
typedef struct epi_mlp epi_mlp;
epi_status epi_mlp_create(epi_ctx *ctx, int n_in, int hidden, uint64_t seed, epi_mlp **out);
void epi_mlp_destroy(epi_mlp *net);
int64_t epi_mlp_num_params(const epi_mlp *net);
/* Inference kernel choice: 0 automatic (tensor cores where they apply),
 * 1 CUDA-core layers, 2 tensor cores (EPI_EUNSUPPORTED for other shapes). */
epi_status epi_mlp_set_forward_path(epi_mlp *net, int path);
int epi_mlp_num_inputs(const epi_mlp *net);
/* FP32 master parameters to / from host memory (epi_mlp_num_params floats);
 * setting them also resets the optimiser's step count. */
epi_status epi_mlp_get_params(const epi_mlp *net, float *host);
epi_status epi_mlp_set_params(epi_mlp *net, const float *host);
/* Input normalisation applied before the first layer: feature f enters as
 * (x_f - shift[f]) * scale[f] (host arrays of n_in floats; defaults 0 and 1).
 * Saved with the network by the bindings; not changed by training steps. */
epi_status epi_mlp_set_input_norm(epi_mlp *net, const float *shift_host, const float *scale_host);
epi_status epi_mlp_get_input_norm(const epi_mlp *net, float *shift_host, float *scale_host);
/* Predictions for `rows` device inputs X [rows][n_in] into device y [rows].
 * With hidden = 256 and n_in <= 32 one fused tensor-core kernel runs the
 * three layers (BF16 operands, FP32 accumulation, activations rounded to
 * BF16 between layers, as in training) and the call waits for it (status
 * EPI_ETIMEOUT if a bounded wait gave up); other shapes run the CUDA-core
 * layers in slices of bounded activation memory, queued on the stream. */
epi_status epi_mlp_forward(epi_mlp *net, const float *X_dev, int64_t rows, float *y_dev);
/* Gradients of the mean squared error against device targets t [rows] into
 * host grad [num_params] (may be NULL); host loss (may be NULL). */
epi_status epi_mlp_gradients(epi_mlp *net, const float *X_dev, const float *t_dev, int64_t rows, float *grad_host,
                             float *loss_host);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay wd) on
 * the mean squared error of the batch; host loss before the step (may be NULL). */
epi_status epi_mlp_train_step(epi_mlp *net, const float *X_dev, const float *t_dev, int64_t rows, float lr,
                              float wd, float *loss_host);

/* Order-5 proposal search.  The exhaustive order-1..3 scores of the dataset
 * (and order 4 with quad_features) are computed (popcount path) on the first
 * proposer call that needs them and kept with the dataset until it is
 * destroyed (4 (n + C(n,2) + C(n,3) [+ C(n,4)]) bytes of device memory;
 * EPI_ENOMEM if the order-4 table would take more than half of the free
 * memory); the top_triples best triples by order-3 MI (ties by rank), listed
 * in rank order, are each joined with every pair of other SNPs; every
 * distinct 5-set of that space (a set holding several of the triples is taken
 * once) is ranked by `net` from its 25 or 30 features (epi_features5), or,
 * with net NULL, by epi_heuristic5 of those features; the best `budget`
 * are counted and scored exactly (Section 2.2 tables, Eq. 1-3 in FP64), and
 * the best top_n by exact MI (ties by lexicographic rank) are written to host
 * out [top_n] (order 5) with their tables in host counts [top_n][2][243]
 * (counts may be NULL).  chunk = candidates ranked per pass (0: 4Mi).  The
 * paper has no counterpart: it searches exhaustively; this call is an
 * approximation whose result is exact only for the sets it proposes. */
typedef struct epi_proposer_opts {
    int top_triples;   /* 1..2^24 (capped at C(n_snps, 3)) */
    int budget;        /* proposals re-scored exactly, 1..2^30: the budget's
                          best distinct candidates by (ranking score desc,
                          candidate index asc), selected by radix select over
                          every ranked score (kept in device memory, 5 bytes
                          per candidate; EPI_ENOMEM if that does not fit);
                          every proposal is scored exactly in FP32 and the
                          4096 best of those again in FP64 */
    int top_n;         /* 1..min(budget, 4096) */
    int64_t chunk;
    int quad_features; /* 0: the 25 features of orders 1-3; 1: the 30
                          features with the four-way scores (a network must
                          then take 30 inputs) */
} epi_proposer_opts;
typedef struct epi_proposer_stats {
    uint64_t candidates;   /* top_triples * C(n_snps - 3, 2) */
    uint64_t kept;         /* distinct sets among them (ranked) */
    uint64_t proposals;    /* sets re-scored exactly */
    double ms_lower, ms_rank, ms_rescore;   /* wall time of the three stages */
    int32_t exact_in_proposals;   /* 1: out is the exact top_n of the proposals
                                     (always for budgets up to 4096; above, when
                                     the FP32 pool margin proves it) */
} epi_proposer_stats;
epi_status epi_proposer_search(epi_dataset *ds, epi_mlp *net, const epi_proposer_opts *opts, epi_result *out,
                               uint32_t *counts, int32_t *n_out, epi_proposer_stats *stats);

/* Fits `net` (25 inputs, or 30 for the features with four-way scores) to
 * rank order-5 sets: on each dataset the space of
 * epi_proposer_search with the given top_triples is built and every row (a
 * candidate 5-set) is labelled by its exact MI (its table counted, Section
 * 2.2, and scored, Eq. 1-3; see `target`), a set holding several of the
 * triples counted once for sampling; inputs are standardised (the
 * normalisation is stored in the network), and `epochs` passes of
 * mini-batch AdamW (cosine decay from lr to lr / 20, weight decay wd) are
 * run; tail_fraction of each batch is drawn from the 4096 best-labelled sets
 * of each dataset, the rest uniformly, from a counter-based generator seeded
 * by `seed`.  The rows stay in device memory (4 n_in + 13 bytes each; EPI_ENOMEM if
 * they do not fit).  Host epoch_loss [epochs] (may be NULL) receives the mean
 * sampled batch loss of each epoch.  The paper has no counterpart. */
typedef struct epi_train_opts {
    int top_triples;
    int epochs;
    int batch;           /* 1..2^20 */
    float lr, wd;
    float tail_fraction; /* 0..1 */
    uint64_t seed;
    int target;          /* 0: standardised ln(MI + 1e-7); 1: 1 for the 4096
                            best-labelled sets of each dataset, else 0 */
} epi_train_opts;
epi_status epi_proposer_train(epi_mlp *net, epi_dataset *const *datasets, int n_ds, const epi_train_opts *opts,
                              float *epoch_loss);

/* Every contingency table of order 2..4 (Section 2.2), its last level
 * counted with one of three instructions, for comparing them (the paper
 * compares popcount implementations the same way, Section 3.1, Table 1):
 * variant 0 the POPC instruction, 1 a 256-entry byte lookup table in shared
 * memory, 2 the binary tensor-core MMA (mma.sync m16n8k256, AND + POPC).
 * Each prefix's genotype table is built once in shared memory and genotype 2
 * of the last SNP comes by subtraction, as in the search.  *checksum
 * receives sum over all tables and cells of count * (1 + cell + 3^k class),
 * the same for every variant; tables (may be NULL) receives every table,
 * host [C(n,k)][2][3^k] in lexicographic rank order (at most 2 GiB); *ms
 * (may be NULL) the kernel's event time. */
epi_status epi_count_variant(epi_dataset *ds, int order, int variant, uint32_t *tables, uint64_t *checksum,
                             double *ms);

/* Test controls of a context (the paper has no counterpart; they exist so
 * that the failure paths can be exercised without faulting a GPU).
 *
 * epi_set_wait_limit: every pipeline wait of the tensor-core counting kernel
 * (a role waiting for another role's stage, accumulator or descriptor) gives
 * up after limit_ns nanoseconds instead of the default 2 s (0 restores the
 * default).  A wait that gives up makes every role leave its loop, wait (with
 * the default limit) for its own copies and MMAs in flight, free tensor
 * memory and return; the search then fails with EPI_ETIMEOUT and the context
 * stays usable.
 *
 * epi_inject_alloc_failure: the device allocation of this context's calls
 * that comes after `after` further successful ones fails as if the device
 * were out of memory (the call returns EPI_ENOMEM and releases what it had
 * taken); it fires once.  A negative value cancels it.
 *
 * epi_set_tc_variant: which tensor-core counting variant this context's
 * searches use (an epi_tc_variant; EPI_TC_AUTO is the default).  Both count
 * exactly and give identical results; EPI_TC_SEPARATE exists so that either
 * variant can be checked on any dataset.  EPI_EINVAL for other values. */
epi_status epi_set_wait_limit(epi_ctx *ctx, uint64_t limit_ns);
epi_status epi_inject_alloc_failure(epi_ctx *ctx, int64_t after);
epi_status epi_set_tc_variant(epi_ctx *ctx, int variant);

/* Rate of the tensor pipe for an MMA the tensor-core counting path issues
 * (tcgen05.mma kind::f8f6f4, operands in shared memory, FP32 accumulation):
 * shape 0 = M128 N128 K32 with E4M3 operands (separate-class variant),
 * shape 1 = M128 N256 K32 with E5M2 operands (combined-class variant);
 * EPI_EINVAL for other shapes.  One CTA per SM issues `stages` (32..2^32)
 * groups of four such MMAs back to back from one thread, with no other work.
 * The paper has no counterpart; this is the roofline's denominator.
 * out[4]: dense rate in TFLOP/s (2 flop per multiply-add, over the launch's
 * event time), multiply-adds per SM clock (over each CTA's own cycle count,
 * averaged), the launch's milliseconds, and the implied SM clock in MHz. */
epi_status epi_tc_rate(epi_ctx *ctx, int shape, int64_t stages, double *out);

/* Timing of the dominant counting kernel.  After epi_profile_begin, every
 * launch of a search's counting kernel is bracketed by CUDA events on the
 * context's stream; epi_profile_end waits for those events and returns their
 * summed duration in milliseconds and the number of bracketed launches. */
epi_status epi_profile_begin(epi_ctx *ctx);
epi_status epi_profile_end(epi_ctx *ctx, double *kernel_ms, int64_t *launches);

/* Wait-cycle trace of the last tensor-core search run while profiling was on
 * (the paper has no counterpart): out[8] receives, averaged over CTAs, the
 * SM cycles the MMA issuer waited for generated prefix tiles [0], for TMA
 * tiles [1] and for a free accumulator [2], the A producers waited for a free
 * stage [3] and for a free accumulator [4], the epilogue waited for a
 * finished accumulator and its row totals [5], the TMA
 * producer waited for a free stage [6], and the MMA issuer's whole loop [7].
 * Zeros when no such search ran.  The value must be read before the context's
 * next search (the scratch memory is reused). */
epi_status epi_profile_waits(epi_ctx *ctx, double *out);

#ifdef __cplusplus
}
#endif

#endif /* EPI_H */
