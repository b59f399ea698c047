/*
 * Plain FP64 CPU oracle for BM25S eager sparse scoring.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the tests, by the smoke
 * check and by the timed CPU baseline of the benchmark; the product path
 * (the CUDA library) never links, loads or calls it, and the two share no
 * code, headers or constants.
 *
 * What it computes, and from where (arXiv 2407.03618, "BM25S: Orders of
 * magnitude faster lexical search via eager sparse scoring"):
 *   - B(Q,D) = sum_i S(q_i, D)                             Sec. 2, "Calculation of BM25"
 *   - S(t,D) = IDF(t) * TF(t,D) / (TF(t,D) + k1 (1 - b + b |D| / Lavg))
 *     with |D| and Lavg counted in tokens                  Sec. 2, "Calculation of BM25"
 *   - IDF(t) = ln((|C| - DF + 0.5) / (DF + 0.5) + 1)       Sec. 2, "Calculation of BM25"
 *   - eager storage of S(t,D) for TF > 0 only (TF = 0 => S = 0)
 *                                                          Sec. 2, "Eager index-time scoring"
 *   - the other four variants (Robertson, ATIRE, BM25L, BM25+) follow the
 *     definitions the paper adopts from Kamphuis et al. 2020 (Sec. 2,
 *     "Alternative BM25 implementations"); the paper prints only Lucene's.
 *   - TF_{l o delta o p} x IDF, which Sec. 2.1 names as the third model whose
 *     non-occurrence score is not zero (Rousseau and Vazirgiannis 2013):
 *     the pivoted length normalisation p (TF / (1 - b + b |D| / Lavg)), then
 *     the lower bound delta (+ delta), then the double logarithm l
 *     (x -> 1 + ln(1 + ln x)), times IDF = ln((|C| + 1) / DF).  Read, as
 *     Sec. 2.1 does, at TF = 0 too: S0 = IDF (1 + ln(1 + ln delta)), defined
 *     for delta > 1/e.
 *   - the non-occurrence score S0(t) = S(t, empty doc) and the shifted
 *     matrix S - S0, with B = sum S_delta + sum S0       Sec. 2.1
 *   - top-k over ALL documents, ties broken by lower doc id
 *                                                          Sec. 2, "Top-k selection"
 *
 * The oracle is lazy and exhaustive: oracle_score_all() evaluates B(Q,D) for
 * every document from TF looked up per document, including TF = 0 terms, so
 * it is an independent check of the eager (shifted, sparse) form that the GPU
 * path implements.  oracle_build() also produces the eager term-major CSC so
 * that structure (TF, DF, |D|, indptr, indices) can be compared bit for bit.
 *
 * Readings taken where the paper is silent:
 *   - a term with DF = 0 has IDF = 0 and S0 = 0 in every variant;
 *   - |D| is the exact token count (no length quantisation);
 *   - duplicate query tokens count once per occurrence (the sum over i);
 *   - an empty query scores 0 everywhere.
 */
#define _GNU_SOURCE /* qsort_r */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LUCENE 0
#define ORC_ROBERTSON 1
#define ORC_ATIRE 2
#define ORC_BM25L 3
#define ORC_BM25PLUS 4
#define ORC_TFLDP 5

/* ---- per-variant formulas (FP64) ------------------------------------- */

/* IDF(t) from |C| = n and DF(t) = df.  Lucene is printed in Sec. 2; the
 * others are the Kamphuis et al. definitions the paper defers to.  DF = 0
 * gives 0 (reading: a term that occurs nowhere contributes nothing). */
double oracle_idf(int variant, double n, double df)
{
    if (df <= 0.0)
        return 0.0;
    switch (variant) {
    case ORC_LUCENE:
        return log((n - df + 0.5) / (df + 0.5) + 1.0);
    case ORC_ROBERTSON:
        return log((n - df + 0.5) / (df + 0.5));
    case ORC_ATIRE:
        return log(n / df);
    case ORC_BM25L:
        return log((n + 1.0) / (df + 0.5));
    case ORC_BM25PLUS:
    case ORC_TFLDP:
        return log((n + 1.0) / df);
    }
    return NAN;
}

/* S(t,D) for one term and one document, TF >= 0 (TF = 0 is the lazy
 * "term absent" case).  len = |D|, lavg = mean |D|.
 *
 * The TF-dependent fraction is 0 when TF = 0 (Sec. 2: an absent term scores
 * 0 in the sparse variants).  It is written out as 0 rather than evaluated,
 * because the normaliser can be 0/0 there: an all-empty corpus has Lavg = 0,
 * and b = 1 on an empty document gives 1 - b + b|D|/Lavg = 0.  BM25L's
 * c = TF / normaliser is 0 at TF = 0 for the same reason. */
double oracle_term_score(int variant, double idf, double tf, double len,
                         double lavg, double k1, double b, double delta)
{
    /* the length normaliser 1 - b + b |D| / Lavg from Sec. 2 */
    double norm = (tf > 0.0) ? 1.0 - b + b * len / lavg : 1.0;
    switch (variant) {
    case ORC_LUCENE:
    case ORC_ROBERTSON:
        return (tf > 0.0) ? idf * tf / (tf + k1 * norm) : 0.0;
    case ORC_ATIRE:
        return (tf > 0.0) ? idf * (k1 + 1.0) * tf / (tf + k1 * norm) : 0.0;
    case ORC_BM25L: {
        double c = (tf > 0.0) ? tf / norm : 0.0;
        return idf * (k1 + 1.0) * (c + delta) / (k1 + c + delta);
    }
    case ORC_BM25PLUS:
        return idf * (((tf > 0.0) ? (k1 + 1.0) * tf / (k1 * norm + tf) : 0.0) + delta);
    case ORC_TFLDP: {
        /* p: pivoted normalisation, delta: lower bound, l: 1 + ln(1 + ln x) */
        double p = (tf > 0.0) ? tf / norm : 0.0;
        double x = p + delta;
        return idf * (1.0 + log(1.0 + log(x)));
    }
    }
    return NAN;
}

/* S0(t) = S(t, empty document): the score a term gets where it does not
 * occur (Sec. 2.1), i.e. S evaluated at TF = 0 (the empty document). */
double oracle_nonoccurrence(int variant, double idf, double k1, double b,
                            double delta)
{
    return oracle_term_score(variant, idf, 0.0, 1.0, 1.0, k1, b, delta);
}

/* ---- index ------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Builds everything the method derives from the corpus.
 *
 * Inputs: tokens[n_tokens], doc_offsets[n_docs + 1] (doc D owns
 * tokens[off[D] .. off[D+1])), vocab size, variant, k1, b, delta.
 *
 * Outputs (caller-allocated):
 *   doc_len[n_docs]            |D| in tokens
 *   *lavg                      mean |D| (FP64)
 *   pair_start[n_docs + 1]     doc-major offsets into the pair arrays
 *   pair_term[cap], pair_tf[cap]   per doc, its distinct terms ascending with TF
 *   df[vocab], idf[vocab], s0[vocab]
 *   indptr[vocab + 1], indices[cap], csc_tf[cap], csc_delta[cap]
 *       term-major CSC of the shifted score S - S0, doc ids ascending
 * cap must be >= n_tokens.  Returns nnz, or -1 on a token outside
 * [0, vocab) or malformed offsets. */
int64_t oracle_build(const int32_t* tokens, int64_t n_tokens,
                     const int64_t* doc_offsets, int64_t n_docs, int32_t vocab,
                     int variant, double k1, double b, double delta,
                     int64_t* doc_len, double* lavg, int64_t* pair_start,
                     int32_t* pair_term, int32_t* pair_tf, int64_t* df,
                     double* idf, double* s0, int64_t* indptr,
                     int32_t* indices, int32_t* csc_tf, double* csc_delta)
{
    if (n_docs < 1 || vocab < 1 || doc_offsets[0] != 0 ||
        doc_offsets[n_docs] != n_tokens)
        return -1;
    for (int64_t i = 0; i < n_tokens; i++)
        if (tokens[i] < 0 || tokens[i] >= vocab)
            return -1;

    /* |D| and Lavg (Sec. 2: lengths in tokens) */
    int64_t total = 0;
    for (int64_t d = 0; d < n_docs; d++) {
        if (doc_offsets[d + 1] < doc_offsets[d])
            return -1;
        doc_len[d] = doc_offsets[d + 1] - doc_offsets[d];
        total += doc_len[d];
    }
    *lavg = (double)total / (double)n_docs;

    /* TF: sort each document's tokens, count runs */
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (n_tokens > 0 ? n_tokens : 1));
    int64_t nnz = 0;
    for (int64_t d = 0; d < n_docs; d++) {
        int64_t lo = doc_offsets[d], len = doc_len[d];
        pair_start[d] = nnz;
        memcpy(buf, tokens + lo, sizeof(int32_t) * len);
        qsort(buf, len, sizeof(int32_t), cmp_i32);
        for (int64_t i = 0; i < len;) {
            int64_t j = i;
            while (j < len && buf[j] == buf[i])
                j++;
            pair_term[nnz] = buf[i];
            pair_tf[nnz] = (int32_t)(j - i);
            nnz++;
            i = j;
        }
    }
    pair_start[n_docs] = nnz;
    free(buf);

    /* DF: number of documents containing the term */
    for (int32_t t = 0; t < vocab; t++)
        df[t] = 0;
    for (int64_t p = 0; p < nnz; p++)
        df[pair_term[p]]++;

    /* IDF and S0 per term */
    for (int32_t t = 0; t < vocab; t++) {
        idf[t] = oracle_idf(variant, (double)n_docs, (double)df[t]);
        s0[t] = (df[t] > 0) ? oracle_nonoccurrence(variant, idf[t], k1, b, delta) : 0.0;
    }

    /* term-major CSC: column t holds the documents containing t, ascending */
    indptr[0] = 0;
    for (int32_t t = 0; t < vocab; t++)
        indptr[t + 1] = indptr[t] + df[t];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * vocab);
    for (int32_t t = 0; t < vocab; t++)
        fill[t] = indptr[t];
    for (int64_t d = 0; d < n_docs; d++) { /* docs in ascending order */
        for (int64_t p = pair_start[d]; p < pair_start[d + 1]; p++) {
            int32_t t = pair_term[p];
            int64_t j = fill[t]++;
            indices[j] = (int32_t)d;
            csc_tf[j] = pair_tf[p];
            csc_delta[j] = oracle_term_score(variant, idf[t], (double)pair_tf[p],
                                             (double)doc_len[d], *lavg, k1, b, delta) -
                           s0[t];
        }
    }
    free(fill);
    return nnz;
}

/* ---- retrieval -------------------------------------------------------- */

/* TF(t, D) from the doc-major pair list (terms ascending within a doc). */
static int32_t lookup_tf(const int64_t* pair_start, const int32_t* pair_term,
                         const int32_t* pair_tf, int64_t d, int32_t t)
{
    int64_t lo = pair_start[d], hi = pair_start[d + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (pair_term[mid] < t)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < pair_start[d + 1] && pair_term[lo] == t)
        return pair_tf[lo];
    return 0;
}

/* Lazy exhaustive B(Q,D) = sum_i S(q_i, D) for every document (Sec. 2),
 * TF = 0 terms included.  q has q_len tokens (duplicates count per
 * occurrence).  Tokens outside [0, vocab) contribute nothing.  If abs_out is
 * not NULL it receives sum_i |S(q_i, D)|, the scale of the rounding error of
 * any summation order. */
void oracle_score_all(const int32_t* q, int64_t q_len, int64_t n_docs,
                      int32_t vocab, int variant, double k1, double b,
                      double delta, const int64_t* doc_len, double lavg,
                      const int64_t* pair_start, const int32_t* pair_term,
                      const int32_t* pair_tf, const double* idf, double* out,
                      double* abs_out)
{
    for (int64_t d = 0; d < n_docs; d++) {
        double s = 0.0, a = 0.0;
        for (int64_t i = 0; i < q_len; i++) {
            int32_t t = q[i];
            if (t < 0 || t >= vocab)
                continue;
            int32_t tf = lookup_tf(pair_start, pair_term, pair_tf, d, t);
            double st = oracle_term_score(variant, idf[t], (double)tf, (double)doc_len[d],
                                          lavg, k1, b, delta);
            s += st;
            a += fabs(st);
        }
        out[d] = s;
        if (abs_out)
            abs_out[d] = a;
    }
}

/* Full ranking: order[0..n) = documents by (score descending, id ascending).
 * -0.0 compares equal to +0.0. */
static int cmp_rank(const void* a, const void* b, void* ctx)
{
    const double* sc = (const double*)ctx;
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    if (sc[x] > sc[y])
        return -1;
    if (sc[x] < sc[y])
        return 1;
    return (x > y) - (x < y);
}

void oracle_rank(const double* scores, int64_t n, int64_t* order)
{
    for (int64_t i = 0; i < n; i++)
        order[i] = i;
    qsort_r(order, n, sizeof(int64_t), cmp_rank, (void*)scores);
}

/* Top-k for a batch of queries: lazy scoring of every document, then a full
 * sort.  Query q owns q_tokens[q_off[q] .. q_off[q+1]).  Writes
 * out_ids[q*k + r], out_scores[q*k + r]; slots r >= n_docs get id -1 and
 * score -inf.  Queries are spread over n_threads POSIX threads. */
typedef struct {
    const int32_t* q_tokens;
    const int64_t* q_off;
    int64_t q_begin, q_end, k, n_docs;
    int32_t vocab;
    int variant;
    double k1, b, delta, lavg;
    const int64_t *doc_len, *pair_start;
    const int32_t *pair_term, *pair_tf;
    const double* idf;
    int64_t* out_ids;
    double* out_scores;
} topk_job;

static void* topk_worker(void* arg)
{
    topk_job* j = (topk_job*)arg;
    double* sc = (double*)malloc(sizeof(double) * j->n_docs);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * j->n_docs);
    for (int64_t q = j->q_begin; q < j->q_end; q++) {
        oracle_score_all(j->q_tokens + j->q_off[q], j->q_off[q + 1] - j->q_off[q],
                         j->n_docs, j->vocab, j->variant, j->k1, j->b, j->delta,
                         j->doc_len, j->lavg, j->pair_start, j->pair_term,
                         j->pair_tf, j->idf, sc, NULL);
        oracle_rank(sc, j->n_docs, order);
        for (int64_t r = 0; r < j->k; r++) {
            if (r < j->n_docs) {
                j->out_ids[q * j->k + r] = order[r];
                j->out_scores[q * j->k + r] = sc[order[r]];
            } else {
                j->out_ids[q * j->k + r] = -1;
                j->out_scores[q * j->k + r] = -INFINITY;
            }
        }
    }
    free(sc);
    free(order);
    return NULL;
}

void oracle_topk(const int32_t* q_tokens, const int64_t* q_off, int64_t n_queries,
                 int64_t k, int64_t n_docs, int32_t vocab, int variant, double k1,
                 double b, double delta, const int64_t* doc_len, double lavg,
                 const int64_t* pair_start, const int32_t* pair_term,
                 const int32_t* pair_tf, const double* idf, int n_threads,
                 int64_t* out_ids, double* out_scores)
{
    if (n_threads < 1)
        n_threads = 1;
    if (n_threads > n_queries)
        n_threads = (int)(n_queries > 0 ? n_queries : 1);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
    topk_job* jobs = (topk_job*)malloc(sizeof(topk_job) * n_threads);
    for (int i = 0; i < n_threads; i++) {
        topk_job* j = &jobs[i];
        j->q_tokens = q_tokens;
        j->q_off = q_off;
        j->q_begin = n_queries * i / n_threads;
        j->q_end = n_queries * (i + 1) / n_threads;
        j->k = k;
        j->n_docs = n_docs;
        j->vocab = vocab;
        j->variant = variant;
        j->k1 = k1;
        j->b = b;
        j->delta = delta;
        j->lavg = lavg;
        j->doc_len = doc_len;
        j->pair_start = pair_start;
        j->pair_term = pair_term;
        j->pair_tf = pair_tf;
        j->idf = idf;
        j->out_ids = out_ids;
        j->out_scores = out_scores;
        pthread_create(&th[i], NULL, topk_worker, j);
    }
    for (int i = 0; i < n_threads; i++)
        pthread_join(th[i], NULL);
    free(th);
    free(jobs);
}
