/*
 * CPU oracle for the exhaustive k-SNP mutual-information search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library: it has its own bit packing, its own enumeration and
 * its own scoring, written plainly so that each step can be checked against
 * the paper by eye.  Nothing here is tuned.
 *
 * What it computes (all sections refer to Ponte-Fernandez et al., "A SIMD
 * algorithm for the detection of epistatic interactions of any order",
 * arXiv 2201.02460):
 *   - genotype tables (Section 2.1, Fig. 2): per SNP, a case subtable and a
 *     control subtable with 3 rows (genotype 0, 1, 2) of 1 bit per
 *     individual, zero padded to whole 64-bit words;
 *   - combination of a table with one more SNP by row-wise AND (Section 2.1,
 *     Listing A.1): row (i*3+j) of the result = row i of the prefix table AND
 *     row j of the SNP table, so the first SNP is the most significant digit;
 *   - the last level fused with the population count (Section 2.2, Listing
 *     A.2): cell (i*3+j) = sum over words of popcount(prefix_i & snp_j);
 *   - mutual information MI = H(X) + H(Y) - H(X,Y) in nats, with
 *     probabilities = count / m over all m individuals and 0 log 0 taken as 0
 *     (Section 2.3, Eq. 1-3).  Evaluated in double precision;
 *   - exhaustive enumeration of every k-subset with the (k-1)-prefix table
 *     computed once and reused for every last SNP (Section 2.4, Algorithm 1).
 *     Subsets are visited in lexicographic order instead of through the
 *     paper's stack; the visited set is the same;
 *   - only the N best combinations are retained (Section 2.4): ordered by MI
 *     descending, equal MI broken by the lexicographically smaller index
 *     tuple.
 *
 * Bit order: bit b of word w of a subtable row is individual 64 w + b of that
 * subtable, where the subtable lists its individuals in input order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EO_OK 0
#define EO_EINVAL 1
#define EO_ENOMEM 2
#define EO_MAX_K 8

/* ------------------------------------------------------------------ */
/* binomial coefficients and lexicographic ranking                     */
/* ------------------------------------------------------------------ */

/* C(n, k); returns UINT64_MAX when the value does not fit in 64 bits. */
uint64_t eo_binom(int64_t n, int64_t k)
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

/* Combination of lexicographic rank r among the k-subsets of [0, n). */
int eo_unrank(int64_t n, int k, uint64_t r, int32_t *out)
{
    if (k < 1 || k > n || r >= eo_binom(n, k)) return EO_EINVAL;
    int64_t c = 0;
    for (int t = 0; t < k; t++) {
        for (;; c++) {
            uint64_t below = eo_binom(n - 1 - c, k - 1 - t);
            if (r < below) break;
            r -= below;
        }
        out[t] = (int32_t)c;
        c++;
    }
    return EO_OK;
}

/* Lexicographic rank of a strictly increasing k-subset of [0, n). */
uint64_t eo_rank(int64_t n, int k, const int32_t *comb)
{
    uint64_t r = 0;
    int64_t start = 0;
    for (int t = 0; t < k; t++) {
        for (int64_t c = start; c < comb[t]; c++) r += eo_binom(n - 1 - c, k - 1 - t);
        start = comb[t] + 1;
    }
    return r;
}

/* Next k-subset in lexicographic order; returns the first position that
 * changed, or -1 after the last subset. */
static int next_comb(int64_t n, int k, int32_t *c)
{
    int t = k - 1;
    while (t >= 0 && c[t] == n - k + t) t--;
    if (t < 0) return -1;
    c[t]++;
    for (int u = t + 1; u < k; u++) c[u] = c[u - 1] + 1;
    return t;
}

/* ------------------------------------------------------------------ */
/* genotype tables                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n, m, m_case, m_ctrl;
    int64_t w_case, w_ctrl;   /* 64-bit words per subtable row */
    int64_t w;                /* w_case + w_ctrl */
    uint64_t *tab;            /* [n][3][w]: case words then control words */
} eo_data;

static int eo_data_build(const uint8_t *geno, const uint8_t *pheno, int64_t n, int64_t m,
                         eo_data *d)
{
    memset(d, 0, sizeof(*d));
    if (n < 1 || m < 1) return EO_EINVAL;
    int64_t m1 = 0;
    for (int64_t i = 0; i < m; i++) {
        if (pheno[i] > 1) return EO_EINVAL;
        m1 += pheno[i];
    }
    for (int64_t i = 0; i < n * m; i++)
        if (geno[i] > 2) return EO_EINVAL;
    d->n = n; d->m = m; d->m_case = m1; d->m_ctrl = m - m1;
    d->w_case = (m1 + 63) / 64;
    d->w_ctrl = (m - m1 + 63) / 64;
    d->w = d->w_case + d->w_ctrl;
    size_t words = (size_t)n * 3 * (size_t)(d->w ? d->w : 1);
    d->tab = (uint64_t *)calloc(words, sizeof(uint64_t));
    if (!d->tab) return EO_ENOMEM;
    for (int64_t s = 0; s < n; s++) {
        uint64_t *t = d->tab + (size_t)s * 3 * d->w;
        int64_t ic = 0, in = 0;
        for (int64_t i = 0; i < m; i++) {
            int g = geno[(size_t)s * m + i];
            int64_t pos;
            if (pheno[i]) pos = ic++;                 /* case subtable */
            else pos = d->w_case * 64 + in++;         /* control subtable */
            t[(size_t)g * d->w + pos / 64] |= (uint64_t)1 << (pos % 64);
        }
    }
    return EO_OK;
}

static void eo_data_free(eo_data *d) { free(d->tab); d->tab = NULL; }

static const uint64_t *snp_rows(const eo_data *d, int64_t s) { return d->tab + (size_t)s * 3 * d->w; }

/* Listing A.1 semantics: out row (i*3+j) = prefix row i AND snp row j, over
 * the case words and the control words alike (both subtables at once). */
static void combine(const uint64_t *prefix, int64_t rows, const uint64_t *snp, int64_t w,
                    uint64_t *out)
{
    for (int64_t i = 0; i < rows; i++)
        for (int j = 0; j < 3; j++)
            for (int64_t x = 0; x < w; x++)
                out[(i * 3 + j) * w + x] = prefix[i * w + x] & snp[j * w + x];
}

/* Listing A.2 semantics: the last combination level is never stored, each
 * AND result is counted at once.  Cell (i*3+j) gets the count of cases and
 * the count of controls separately. */
static void combine_and_popcnt(const eo_data *d, const uint64_t *prefix, int64_t rows,
                               const uint64_t *snp, uint32_t *ct_case, uint32_t *ct_ctrl)
{
    for (int64_t i = 0; i < rows; i++)
        for (int j = 0; j < 3; j++) {
            uint32_t a = 0, b = 0;
            for (int64_t x = 0; x < d->w_case; x++)
                a += (uint32_t)__builtin_popcountll(prefix[i * d->w + x] & snp[j * d->w + x]);
            for (int64_t x = d->w_case; x < d->w; x++)
                b += (uint32_t)__builtin_popcountll(prefix[i * d->w + x] & snp[j * d->w + x]);
            ct_case[i * 3 + j] = a;
            ct_ctrl[i * 3 + j] = b;
        }
}

/* ------------------------------------------------------------------ */
/* mutual information, Eq. (1)-(3)                                     */
/* ------------------------------------------------------------------ */

static double plogp(double p) { return p > 0.0 ? p * log(p) : 0.0; }

/* MI in nats of a 3^k x 2 contingency table; m = total individuals. */
double eo_mi(const uint32_t *ct_case, const uint32_t *ct_ctrl, int64_t cells, int64_t m)
{
    double h_x = 0.0, h_xy = 0.0, h_y;
    int64_t m1 = 0, m0 = 0;
    for (int64_t c = 0; c < cells; c++) { m1 += ct_case[c]; m0 += ct_ctrl[c]; }
    for (int64_t c = 0; c < cells; c++) {
        double p_case = (double)ct_case[c] / (double)m;
        double p_ctrl = (double)ct_ctrl[c] / (double)m;
        double p_any = (double)(ct_case[c] + ct_ctrl[c]) / (double)m;
        h_xy -= plogp(p_case) + plogp(p_ctrl);
        h_x -= plogp(p_any);
    }
    h_y = -(plogp((double)m1 / (double)m) + plogp((double)m0 / (double)m));
    return h_x + h_y - h_xy;
}

/* ------------------------------------------------------------------ */
/* public table calls                                                  */
/* ------------------------------------------------------------------ */

static int64_t pow3(int k) { int64_t r = 1; while (k-- > 0) r *= 3; return r; }

static int valid_comb(int64_t n, int k, const int32_t *c)
{
    for (int t = 0; t < k; t++) {
        if (c[t] < 0 || c[t] >= n) return 0;
        if (t && c[t] <= c[t - 1]) return 0;
    }
    return 1;
}

/* Prefix table of the first t SNPs of c (t >= 1) into buf (3^t rows). */
static void build_prefix(const eo_data *d, const int32_t *c, int t, uint64_t *buf, uint64_t *tmp)
{
    memcpy(buf, snp_rows(d, c[0]), sizeof(uint64_t) * 3 * d->w);
    int64_t rows = 3;
    for (int u = 1; u < t; u++) {
        combine(buf, rows, snp_rows(d, c[u]), d->w, tmp);
        rows *= 3;
        memcpy(buf, tmp, sizeof(uint64_t) * rows * d->w);
    }
}

/* Full genotype table (3^k rows, each case words then control words, 64-bit
 * LSB-first) of one combination; out holds 3^k * (w_case + w_ctrl) words.
 * w_out receives (w_case, w_ctrl). */
int eo_genotype_table(const uint8_t *geno, const uint8_t *pheno, int64_t n, int64_t m, int k,
                      const int32_t *comb, uint64_t *out, int64_t *w_out)
{
    eo_data d;
    if (k < 1 || k > EO_MAX_K || !valid_comb(n, k, comb)) return EO_EINVAL;
    int rc = eo_data_build(geno, pheno, n, m, &d);
    if (rc) return rc;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * pow3(k) * d.w);
    if (!tmp) { eo_data_free(&d); return EO_ENOMEM; }
    build_prefix(&d, comb, k, out, tmp);
    w_out[0] = d.w_case; w_out[1] = d.w_ctrl;
    free(tmp);
    eo_data_free(&d);
    return EO_OK;
}

/* Contingency tables of `count` combinations; out is [count][2][3^k] with
 * index 0 = cases and 1 = controls, cell x = sum_t g_t 3^(k-1-t). */
int eo_tables(const uint8_t *geno, const uint8_t *pheno, int64_t n, int64_t m, int k,
              const int32_t *combs, int64_t count, uint32_t *out)
{
    eo_data d;
    if (k < 1 || k > EO_MAX_K || count < 0) return EO_EINVAL;
    for (int64_t i = 0; i < count; i++)
        if (!valid_comb(n, k, combs + i * k)) return EO_EINVAL;
    int rc = eo_data_build(geno, pheno, n, m, &d);
    if (rc) return rc;
    int64_t cells = pow3(k);
    uint64_t *ones = (uint64_t *)malloc(sizeof(uint64_t) * d.w);
    uint64_t *pre = (uint64_t *)malloc(sizeof(uint64_t) * (cells / 3) * 3 * d.w + 8);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (cells / 3) * 3 * d.w + 8);
    if (!ones || !pre || !tmp) { free(ones); free(pre); free(tmp); eo_data_free(&d); return EO_ENOMEM; }
    for (int64_t x = 0; x < d.w; x++) ones[x] = ~(uint64_t)0;
    for (int64_t i = 0; i < count; i++) {
        const int32_t *c = combs + i * k;
        const uint64_t *prefix = ones;
        int64_t rows = 1;
        if (k > 1) { build_prefix(&d, c, k - 1, pre, tmp); prefix = pre; rows = cells / 3; }
        combine_and_popcnt(&d, prefix, rows, snp_rows(&d, c[k - 1]),
                           out + (size_t)i * 2 * cells, out + (size_t)i * 2 * cells + cells);
    }
    free(ones); free(pre); free(tmp);
    eo_data_free(&d);
    return EO_OK;
}

/* ------------------------------------------------------------------ */
/* exhaustive search with top-N retention                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double mi;
    int32_t c[EO_MAX_K];
} eo_rec;

static int k_glob_cmp_k = 0;

/* 1 when a ranks before b: larger MI first, then lexicographically smaller. */
static int better(const eo_rec *a, const eo_rec *b, int k)
{
    if (a->mi != b->mi) return a->mi > b->mi;
    for (int t = 0; t < k; t++)
        if (a->c[t] != b->c[t]) return a->c[t] < b->c[t];
    return 0;
}

/* bounded heap whose root is the worst retained record */
typedef struct { eo_rec *v; int64_t size, cap; int k; } eo_heap;

static void heap_push(eo_heap *h, const eo_rec *r)
{
    if (h->size < h->cap) {
        int64_t i = h->size++;
        h->v[i] = *r;
        while (i > 0) {
            int64_t p = (i - 1) / 2;
            if (!better(&h->v[p], &h->v[i], h->k)) break;   /* parent already worse */
            eo_rec t = h->v[p]; h->v[p] = h->v[i]; h->v[i] = t; i = p;
        }
        return;
    }
    if (!better(r, &h->v[0], h->k)) return;
    h->v[0] = *r;
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, rr = l + 1, w = i;
        if (l < h->size && better(&h->v[w], &h->v[l], h->k)) w = l;
        if (rr < h->size && better(&h->v[w], &h->v[rr], h->k)) w = rr;
        if (w == i) break;
        eo_rec t = h->v[w]; h->v[w] = h->v[i]; h->v[i] = t; i = w;
    }
}

static int rec_cmp(const void *a, const void *b)
{
    const eo_rec *x = (const eo_rec *)a, *y = (const eo_rec *)b;
    if (better(x, y, k_glob_cmp_k)) return -1;
    if (better(y, x, k_glob_cmp_k)) return 1;
    return 0;
}

/* Searches the combinations of lexicographic rank in [rank_begin, rank_end)
 * (rank_end is clipped to C(n,k)) and returns the best top_n of them, sorted.
 * out_combs: [top_n][k]; out_mi: [top_n]; out_counts (may be NULL):
 * [top_n][2][3^k]; *n_out = number of records written.  threads <= 0 uses
 * the OpenMP default. */
int eo_search(const uint8_t *geno, const uint8_t *pheno, int64_t n, int64_t m, int k,
              int64_t top_n, uint64_t rank_begin, uint64_t rank_end, int threads,
              int32_t *out_combs, double *out_mi, uint32_t *out_counts, int64_t *n_out)
{
    eo_data d;
    *n_out = 0;
    if (k < 1 || k > EO_MAX_K || k > n || top_n < 1) return EO_EINVAL;
    uint64_t total = eo_binom(n, k);
    if (total == UINT64_MAX) return EO_EINVAL;
    if (rank_end > total) rank_end = total;
    if (rank_begin >= rank_end) return EO_OK;
    int rc = eo_data_build(geno, pheno, n, m, &d);
    if (rc) return rc;
    const int64_t cells = pow3(k);
    const uint64_t span = rank_end - rank_begin;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = threads > 0 ? threads : omp_get_max_threads();
#endif
    uint64_t nchunks = (uint64_t)nthreads * 64;
    if (nchunks > span) nchunks = span;
    eo_heap *heaps = (eo_heap *)calloc((size_t)nthreads, sizeof(eo_heap));
    if (!heaps) { eo_data_free(&d); return EO_ENOMEM; }
    int fail = 0;
    for (int t = 0; t < nthreads; t++) {
        heaps[t].v = (eo_rec *)malloc(sizeof(eo_rec) * (size_t)top_n);
        heaps[t].cap = top_n; heaps[t].k = k;
        if (!heaps[t].v) fail = 1;
    }
    if (!fail) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            eo_heap *h = &heaps[tid];
            /* g[t] = genotype table of the first t SNPs; g[0] = all ones */
            uint64_t *g[EO_MAX_K];
            uint64_t *mem = (uint64_t *)malloc(sizeof(uint64_t) * d.w * (size_t)(2 * cells) + 64);
            uint32_t *ct = (uint32_t *)malloc(sizeof(uint32_t) * 2 * cells);
            if (mem && ct) {
                uint64_t *p = mem;
                for (int t = 0; t < k; t++) { g[t] = p; p += pow3(t) * d.w; }
                for (int64_t x = 0; x < d.w; x++) g[0][x] = ~(uint64_t)0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
                for (int64_t ch = 0; ch < (int64_t)nchunks; ch++) {
                    uint64_t r0 = rank_begin + span / nchunks * ch + (ch < (int64_t)(span % nchunks) ? ch : span % nchunks);
                    uint64_t len = span / nchunks + ((uint64_t)ch < span % nchunks ? 1 : 0);
                    int32_t c[EO_MAX_K];
                    eo_unrank(n, k, r0, c);
                    int changed = 0;      /* first position whose SNP changed */
                    for (uint64_t it = 0; it < len; it++) {
                        /* Algorithm 1: rebuild only the prefix tables whose
                         * SNPs changed, then count against the last SNP */
                        for (int t = changed + 1; t < k; t++)
                            combine(g[t - 1], pow3(t - 1), snp_rows(&d, c[t - 1]), d.w, g[t]);
                        combine_and_popcnt(&d, g[k - 1], pow3(k - 1), snp_rows(&d, c[k - 1]),
                                           ct, ct + cells);
                        eo_rec rec;
                        rec.mi = eo_mi(ct, ct + cells, cells, m);
                        memset(rec.c, 0, sizeof(rec.c));
                        memcpy(rec.c, c, sizeof(int32_t) * k);
                        heap_push(h, &rec);
                        changed = next_comb(n, k, c);
                        if (changed < 0) break;
                    }
                }
            } else {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                fail = 1;
            }
            free(mem); free(ct);
        }
    }
    if (!fail) {
        int64_t all = 0;
        for (int t = 0; t < nthreads; t++) all += heaps[t].size;
        eo_rec *v = (eo_rec *)malloc(sizeof(eo_rec) * (size_t)(all ? all : 1));
        if (!v) fail = 1;
        else {
            int64_t o = 0;
            for (int t = 0; t < nthreads; t++) {
                memcpy(v + o, heaps[t].v, sizeof(eo_rec) * heaps[t].size);
                o += heaps[t].size;
            }
            k_glob_cmp_k = k;
            qsort(v, (size_t)all, sizeof(eo_rec), rec_cmp);
            int64_t keep = all < top_n ? all : top_n;
            for (int64_t i = 0; i < keep; i++) {
                memcpy(out_combs + i * k, v[i].c, sizeof(int32_t) * k);
                out_mi[i] = v[i].mi;
            }
            if (out_counts && keep) {
                int32_t *cs = (int32_t *)malloc(sizeof(int32_t) * k * keep);
                if (cs) {
                    for (int64_t i = 0; i < keep; i++) memcpy(cs + i * k, v[i].c, sizeof(int32_t) * k);
                    eo_tables(geno, pheno, n, m, k, cs, keep, out_counts);
                    free(cs);
                } else fail = 1;
            }
            *n_out = keep;
            free(v);
        }
    }
    for (int t = 0; t < nthreads; t++) free(heaps[t].v);
    free(heaps);
    eo_data_free(&d);
    return fail ? EO_ENOMEM : EO_OK;
}

/* number of OpenMP threads the search uses by default */
int eo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
