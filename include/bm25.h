/*
 * bm25.h -- C ABI of libbm25gpu, a GB300 (sm_103a) implementation of the
 * eager sparse scoring of BM25S (arXiv 2407.03618).
 *
 * The method (Sec. 2): every score S(t,D) a future query token could need is
 * computed at index time and stored in a sparse term-major matrix; a query is
 * answered by slicing its tokens' columns, summing them into per-document
 * scores and keeping the top k.  BM25L and BM25+ store the shifted score
 * S(t,D) - S0(t) and add the per-query constant sum_i S0(q_i) back (Sec. 2.1).
 *
 * Conventions for every entry point:
 *   - Return value: BM25_OK (0) or a negative bm25_status.  On failure a
 *     message is available from bm25_last_error() on the calling thread.
 *   - Pointers are DEVICE pointers (cudaMalloc / torch CUDA memory on the
 *     index's device) unless the entry point's name ends in _host or the
 *     argument is documented as host memory.
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Device
 *     work is enqueued on it; functions return before it finishes unless
 *     stated otherwise.
 *   - The caller owns every array it passes in.  The library owns an index
 *     (and a workspace) until the matching *_free call.
 *   - Errors found by kernels (a token id outside [0, vocab), malformed
 *     offsets) are recorded in a per-index device status word and reported
 *     by bm25_sync_status(); host-side argument checks fail immediately with
 *     BM25_E_INVALID and launch nothing.
 *
 * Variant formulas (K_D = 1 - b + b |D| / Lavg, |D| and Lavg in tokens):
 *   LUCENE     IDF = ln((N - DF + 0.5)/(DF + 0.5) + 1), S = IDF TF/(TF + k1 K_D)   (Sec. 2)
 *   ROBERTSON  IDF = ln((N - DF + 0.5)/(DF + 0.5)),     S as Lucene
 *   ATIRE      IDF = ln(N / DF),                         S = IDF (k1+1) TF/(TF + k1 K_D)
 *   BM25L      IDF = ln((N + 1)/(DF + 0.5)), c = TF/K_D, S = IDF (k1+1)(c + delta)/(k1 + c + delta)
 *   BM25PLUS   IDF = ln((N + 1)/DF),                     S = IDF ((k1+1) TF/(k1 K_D + TF) + delta)
 *   TFLDP      IDF = ln((N + 1)/DF), p = TF/K_D,         S = IDF (1 + ln(1 + ln(p + delta)))
 * (Robertson .. BM25PLUS as the paper adopts them from Kamphuis et al. 2020,
 * Sec. 2 "Alternative BM25 implementations"; TFLDP is TF_{l o delta o p} x
 * IDF of Rousseau and Vazirgiannis 2013, which Sec. 2.1 names among the
 * models with a non-zero score at TF = 0: pivoted normalisation, lower
 * bound delta, double logarithm; k1 is unused, delta > 1/e).  A term with
 * DF = 0 has IDF = 0 and S0 = 0.
 */
#ifndef BM25_GPU_H
#define BM25_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bm25_index bm25_index;
typedef struct bm25_workspace bm25_workspace;
typedef struct bm25_vocab bm25_vocab;

enum bm25_variant {
    BM25_LUCENE = 0,
    BM25_ROBERTSON = 1,
    BM25_ATIRE = 2,
    BM25_L = 3,
    BM25_PLUS = 4,
    BM25_TFLDP = 5   /* TF_{l o delta o p} x IDF */
};

enum bm25_status {
    BM25_OK = 0,
    BM25_E_INVALID = -1,     /* bad argument (host-side check) */
    BM25_E_TOKEN_RANGE = -2, /* a token id outside [0, vocab) or malformed offsets */
    BM25_E_OOM = -3,         /* device allocation failed */
    BM25_E_CUDA = -4,        /* a CUDA runtime call failed */
    BM25_E_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    BM25_PENDING = 1         /* bm25_server_poll: the request has not finished yet */
};

/* Accumulator strategies for retrieval.  A query's accumulator is chosen by
 * the number of postings in its columns (sum of DF over its tokens):
 *   SMEM_TILED  every query on the doc-tiled path: FP32 accumulators for one
 *               doc tile at a time in shared memory, one work item per
 *               (doc tile, query), a cross-tile merge.
 *   AUTO        queries with at most dense_max_postings postings on the dense
 *               path, the rest tiled.
 *   L2_DENSE    as AUTO with the bound raised to at least 2^19 postings.
 * The dense path gives each in-flight query (one CTA) a dense FP32 vector of
 * n_docs accumulators in device memory; only the sectors the query touches
 * are brought in, and they stay in L2 while it runs.  It allocates
 * min(2 * SMs, 2 GiB / (4 n_docs)) such vectors per workspace and is off
 * when none fits. */
enum bm25_accumulator {
    BM25_ACC_UNSET = 0,      /* in a plan being set or passed: keep the current choice */
    BM25_ACC_AUTO = 1,
    BM25_ACC_SMEM_TILED = 2,
    BM25_ACC_L2_DENSE = 3
};

/* Upper bound on min(k, n_docs) for one retrieval call. */
#define BM25_MAX_K 4096

/* How retrieval runs a query batch.  Results do not depend on the plan
 * (beyond the order of FP32 additions); only speed does.  Zero fields take
 * the library's defaults. */
typedef struct bm25_plan {
    int32_t accumulator;        /* enum bm25_accumulator */
    int32_t tile_docs;          /* doc-tile width: a multiple of 1024 in [1024, 49152]
                                   (default 6144) */
    int32_t block_threads;      /* consumer threads per CTA of the tiled kernel: 128, 192,
                                   256 or 512 (default 256; one producer warp is added) */
    int32_t dense_max_postings; /* dense-path bound for AUTO / L2_DENSE, in [0, 2^22]
                                   (default 4096) */
    int32_t stage_entries;      /* packed postings per shared-memory staging buffer of the
                                   tiled kernel: a multiple of 64 in [128, 8192] (default 1536) */
    int32_t stages;             /* staging buffers in its ring, in [2, 8] (default 2) */
} bm25_plan;

/* ------------------------------------------------------------------ index */

/* Eager index build (Sec. 2 "Eager index-time scoring", "Efficient Matrix
 * Sparsity"; Sec. 2.1 for the shift).
 *
 *   token_ids[n_tokens]    int32, device.  Document D owns
 *                          token_ids[doc_offsets[D] .. doc_offsets[D+1]).
 *   doc_offsets[n_docs+1]  int64, device, non-decreasing, doc_offsets[0] = 0,
 *                          doc_offsets[n_docs] = n_tokens.  Empty documents
 *                          are allowed and count in N.
 *   vocab                  number of term ids; every token must be in [0, vocab).
 *   variant                enum bm25_variant.
 *   k1 >= 0, 0 <= b <= 1, delta >= 0 (delta is used by BM25L, BM25PLUS and
 *                          TFLDP; BM25L also needs k1 + delta > 0, TFLDP
 *                          delta > 1/e).
 *   n_docs in [1, 2^31 - 2], n_tokens in [0, 2^31 - 2].
 *
 * Computes |D|, Lavg (FP64), TF per distinct (term, doc) pair, DF, IDF and
 * S0 per term (FP64), and the term-major CSC: indptr[vocab+1] (int64),
 * indices[nnz] (int32 doc ids, strictly ascending within a term), data[nnz]
 * (FP32 S(t,D) - S0(t)).  Stream-ordered; synchronises `cuda_stream` once to
 * learn nnz and returns after the build has been enqueued (the index is usable
 * on `cuda_stream` at once and on other streams after that stream syncs).
 * Returns BM25_E_TOKEN_RANGE (and no index) if a token or offset is invalid. */
int bm25_index_build(const int32_t* token_ids, int64_t n_tokens,
                     const int64_t* doc_offsets, int64_t n_docs, int32_t vocab,
                     int variant, double k1, double b, double delta,
                     void* cuda_stream, bm25_index** out);

/* Same as bm25_index_build with token_ids and doc_offsets in HOST memory
 * (pinned memory makes the copies asynchronous).  Copies them to the current
 * device on `cuda_stream`, builds, and returns once the build has finished. */
int bm25_index_build_host(const int32_t* token_ids, int64_t n_tokens,
                          const int64_t* doc_offsets, int64_t n_docs, int32_t vocab,
                          int variant, double k1, double b, double delta,
                          void* cuda_stream, bm25_index** out);

/* Scalars of an index.  Any output pointer may be NULL.  Host memory. */
int bm25_index_info(const bm25_index* index, int64_t* n_docs, int64_t* n_tokens,
                    int64_t* nnz, int32_t* vocab, int* variant, double* k1,
                    double* b, double* delta, double* lavg);

/* Copies the index's arrays to HOST memory; any pointer may be NULL.
 *   indptr[vocab+1] int64, indices[nnz] int32, data[nnz] float (S - S0),
 *   tf[nnz] int32, df[vocab] int32, doc_len[n_docs] int32,
 *   idf[vocab] double, s0[vocab] double.
 * Synchronous.  This is the save path of a checkpoint (see bm25_index_import). */
int bm25_index_export(const bm25_index* index, int64_t* indptr, int32_t* indices,
                      float* data, int32_t* tf, int32_t* df, int32_t* doc_len,
                      double* idf, double* s0);

/* Rebuilds an index on the current device from arrays previously exported
 * (HOST memory, layouts as in bm25_index_export; tf may be NULL, then TF is
 * stored as 0).  lavg and the parameters are taken as given.  Synchronous. */
int bm25_index_import(int64_t n_docs, int64_t n_tokens, int64_t nnz, int32_t vocab,
                      int variant, double k1, double b, double delta, double lavg,
                      const int64_t* indptr, const int32_t* indices, const float* data,
                      const int32_t* tf, const int32_t* df, const int32_t* doc_len,
                      const double* idf, const double* s0, bm25_index** out);

/* Synchronises `cuda_stream`, then returns and clears the first error any
 * kernel recorded for this index since the last call (BM25_OK if none). */
int bm25_sync_status(const bm25_index* index, void* cuda_stream);

/* Releases the index and its device memory.  Its default workspace (the
 * retrieval scratch of bm25_retrieve and the _host entry points) is kept, one
 * per device, for the next index's first call, so that building and dropping
 * indexes in a loop allocates that scratch once; bm25_release_cached() frees
 * it.  The caller must make sure no work using the index is still in flight.
 * NULL is a no-op. */
void bm25_index_free(bm25_index* index);

/* Frees the retrieval scratch kept from freed indexes (see bm25_index_free)
 * on every device.  No index of this process may be running a call. */
void bm25_release_cached(void);

/* -------------------------------------------------------------- retrieval */

/* Batched top-k retrieval (Sec. 2 "Assigning Query Scores": slice the query
 * tokens' columns and sum them; "Top-k selection").
 *
 *   query_tokens[n_query_tokens]  int32, device.  Query q owns
 *                 query_tokens[query_offsets[q] .. query_offsets[q+1]).
 *                 A token repeated in a query counts once per occurrence.
 *   query_offsets[n_queries+1]  int64, device, non-decreasing, starting at 0
 *                 and ending at n_query_tokens (checked on the device:
 *                 violations record BM25_E_TOKEN_RANGE and the offending
 *                 ranges are clamped).
 *   k >= 1.  Let k' = min(k, n_docs); k' <= BM25_MAX_K.
 *   out_ids[n_queries*k] int32 and out_scores[n_queries*k] float, device.
 *
 * Row q of the outputs holds the k' documents with the highest B(Q,D),
 * sorted by score descending and doc id ascending among equal scores
 * (documents the query does not touch score exactly sum_i S0(q_i) and are
 * eligible like any other).  Scores are B(Q,D) including the shift of
 * Sec. 2.1.  Slots k' .. k-1 get id -1 and score -inf.  A token id outside
 * [0, vocab) contributes nothing and records BM25_E_TOKEN_RANGE (see
 * bm25_sync_status).  Asynchronous on `cuda_stream`.  Uses the index's
 * default workspace, so calls on one index must not overlap on the device
 * (serialise them on one stream, or use bm25_retrieve_ws). */
int bm25_retrieve(const bm25_index* index, const int32_t* query_tokens,
                  int64_t n_query_tokens, const int64_t* query_offsets,
                  int32_t n_queries, int32_t k, int32_t* out_ids, float* out_scores,
                  void* cuda_stream);

/* bm25_retrieve with query_tokens, query_offsets, out_ids and out_scores in
 * HOST memory (pinned memory makes the copies asynchronous).  Copies the
 * queries in, retrieves, copies the results out and returns when they are in
 * host memory.  query_offsets[0] must be 0; n_query_tokens =
 * query_offsets[n_queries]. */
int bm25_retrieve_host(const bm25_index* index, const int32_t* query_tokens,
                       const int64_t* query_offsets, int32_t n_queries, int32_t k,
                       int32_t* out_ids, float* out_scores, void* cuda_stream);

/* A workspace holds the scratch memory of retrieval and grows on demand.
 * bm25_workspace_create sizes it for a call of max_queries queries,
 * max_query_tokens tokens and k_max = max_k under the index's current plan
 * (synchronous).  One workspace serves one call at a time; calls with
 * different workspaces may overlap on the device. */
int bm25_workspace_create(const bm25_index* index, int32_t max_queries,
                          int64_t max_query_tokens, int32_t max_k,
                          bm25_workspace** out);
void bm25_workspace_free(bm25_workspace* ws);

/* Grows `ws` to what one call with these sizes and this plan (HOST pointer;
 * NULL = the index's plan) needs, so that the call itself allocates nothing:
 * do this before capturing the call in a CUDA graph.  A call made during
 * stream capture that would need to grow the workspace fails with
 * BM25_E_INVALID instead.  May enqueue an initialisation kernel on
 * `cuda_stream`. */
int bm25_workspace_reserve(bm25_workspace* ws, const bm25_index* index,
                           int32_t n_queries, int64_t n_query_tokens, int32_t k_max,
                           const bm25_plan* plan, void* cuda_stream);

/* bm25_retrieve with an explicit workspace and plan (HOST pointer; NULL =
 * the index's plan).  Calls with different workspaces may overlap on the
 * device. */
int bm25_retrieve_ws(const bm25_index* index, bm25_workspace* ws,
                     const int32_t* query_tokens, int64_t n_query_tokens,
                     const int64_t* query_offsets, int32_t n_queries, int32_t k,
                     int32_t* out_ids, float* out_scores, const bm25_plan* plan,
                     void* cuda_stream);

/* The general form of bm25_retrieve: queries with different k in one call,
 * an explicit workspace (NULL = the index's default) and plan (HOST pointer,
 * NULL = the index's plan).
 *   query_k[n_queries]  int32, device, each in [1, k_max]; NULL = k_max for
 *                       every query.  An entry outside that range records
 *                       BM25_E_INVALID in the status word and is clamped.
 *   out_ids / out_scores  [n_queries * k_max], device; row q is k_max wide and
 *                       holds query q's min(k_q, n_docs) results, then -1 /
 *                       -inf.
 * Other arguments, results and errors as in bm25_retrieve.  The batch runs
 * in one pass per sub-batch (queries are split only when the tiled path's
 * candidate buffer would exceed 2 GiB). */
int bm25_retrieve_batch(const bm25_index* index, bm25_workspace* ws,
                        const int32_t* query_tokens, int64_t n_query_tokens,
                        const int64_t* query_offsets, int32_t n_queries,
                        const int32_t* query_k, int32_t k_max, int32_t* out_ids,
                        float* out_scores, const bm25_plan* plan, void* cuda_stream);

/* Retrieval that allocates nothing, for callers that cannot call cudaMalloc
 * at this point: a real-time serving loop with a fixed memory budget (an
 * allocation may synchronise the device), a process whose device memory is
 * owned by another allocator.  It still calls the CUDA runtime, so it must
 * not be called from a CUDA host function or stream callback.  The paper has
 * no counterpart; it is an operational variant of bm25_retrieve (same
 * arguments, same results up to the order of FP32 additions).
 *
 * Its scratch is one file-scope device array of 16 MiB that every GPU
 * loading the library holds until the process exits.  Every query takes the
 * doc-tiled path.  A batch whose scratch (about 40 bytes per query, 4 per
 * query token and doc-tile boundary, 4 per query and doc tile, 8 per query,
 * doc tile and k' candidate slot) exceeds 16 MiB fails with BM25_E_INVALID;
 * split it.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture.  That address is kept, so
 * the library must not be used across a cudaDeviceReset.  Every call shares
 * the array: calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller. */
int bm25_retrieve_noalloc(const bm25_index* index, const int32_t* query_tokens,
                          int64_t n_query_tokens, const int64_t* query_offsets,
                          int32_t n_queries, int32_t k, int32_t* out_ids,
                          float* out_scores, void* cuda_stream);

/* Sets / reads the index's default plan (HOST pointers).  Zero fields of a
 * plan being set keep the current values; an invalid field fails with
 * BM25_E_INVALID and changes nothing. */
int bm25_index_set_plan(bm25_index* index, const bm25_plan* plan);
int bm25_index_get_plan(const bm25_index* index, bm25_plan* plan);

/* Times retrieval of a sample batch (device arrays, as in bm25_retrieve,
 * with one k for all queries) under candidate plans and makes the fastest
 * the index's plan.  Candidates: tile widths 6144, 7168, 8192, 10240 and
 * 12288 with every query tiled and the default threads and staging ring,
 * then 128, 192, 256 and 512 consumer threads at the best width, then
 * staging rings of 2 x 512, 2 x 1024, 3 x 1024, 2 x 1536 and 2 x 2048 postings with
 * the best of those, then dense-path bounds of 2048 .. 32768 postings (the
 * accumulator per query-length bucket).  Each step tries the library's default first, and a
 * later candidate replaces the best so far only when more than 1 % faster, so
 * that timing noise does not move the plan between runs.  Each candidate
 * runs once untimed and twice timed (CUDA events on `cuda_stream`); the best
 * of the two counts.  Synchronous; allocates its own scratch.  Results of
 * retrieval do not depend on the plan.
 *   best                 the chosen plan (HOST); best_ms its time (may be NULL).
 *   tried / tried_ms     optional HOST arrays of tried_cap entries: every
 *                        candidate timed, in order; *n_tried their number. */
int bm25_autotune(bm25_index* index, const int32_t* query_tokens, int64_t n_query_tokens,
                  const int64_t* query_offsets, int32_t n_queries, int32_t k,
                  void* cuda_stream, bm25_plan* best, double* best_ms, bm25_plan* tried,
                  double* tried_ms, int32_t tried_cap, int32_t* n_tried);

/* -------------------------------------------------------------- tokenizer */

/* Text to term ids on the device (Sec. 2 "Tokenization": split with the
 * pattern (?u)\b\w\w+\b, remove stopwords, map each distinct word to an
 * integer id).  Read on UTF-8 bytes: ASCII letters, digits and '_' and every
 * byte of a non-ASCII character are word characters, ASCII letters are
 * lowercased, a token is a maximal run of word bytes inside one text with at
 * least two characters, and a token equal to a stopword is dropped.  (The
 * Snowball stemmer the paper offers as an option is not provided.)
 *
 * bm25_tokenize_corpus: text[n_bytes] (device bytes) holds n_docs texts,
 * doc d at text[doc_offsets[d] .. doc_offsets[d+1]) (device int64, starting
 * at 0 and ending at n_bytes); stopwords (HOST bytes, word i at
 * stopwords[stop_offsets[i] .. stop_offsets[i+1]), any case) may be NULL
 * with n_stopwords = 0.  Writes the corpus's term ids to token_ids (device,
 * capacity entries; n_bytes / 2 + 1 always suffices) and
 * token_offsets[n_docs+1] (device int64: doc d owns token_ids[offsets[d] ..
 * offsets[d+1])) — the inputs bm25_index_build takes — sets *n_tokens
 * (host), and returns a vocabulary: ids are given in order of first
 * occurrence.  If the tokens exceed capacity, returns BM25_E_INVALID with
 * *n_tokens set.  Words are told apart by a 64-bit hash checked against
 * their bytes; two different words with the same hash fail with
 * BM25_E_INVALID.  Synchronous.
 *
 * bm25_tokenize_queries: the same split with the vocabulary's stopwords;
 * tokens the vocabulary does not know are dropped; token_offsets[n_texts+1].
 *
 * bm25_vocab_export: the words (lowercased bytes, HOST, n_bytes from
 * bm25_vocab_info) in id order and word_offsets[n_words+1] (HOST); either
 * may be NULL. */
int bm25_tokenize_corpus(const uint8_t* text, int64_t n_bytes, const int64_t* doc_offsets,
                         int64_t n_docs, const uint8_t* stopwords, const int64_t* stop_offsets,
                         int32_t n_stopwords, int32_t* token_ids, int64_t capacity,
                         int64_t* token_offsets, int64_t* n_tokens, bm25_vocab** vocab,
                         void* cuda_stream);
int bm25_tokenize_queries(const bm25_vocab* vocab, const uint8_t* text, int64_t n_bytes,
                          const int64_t* offsets, int64_t n_texts, int32_t* token_ids,
                          int64_t capacity, int64_t* token_offsets, int64_t* n_tokens,
                          void* cuda_stream);
int bm25_vocab_info(const bm25_vocab* vocab, int64_t* n_words, int64_t* n_bytes);
int bm25_vocab_export(const bm25_vocab* vocab, uint8_t* words, int64_t* word_offsets);
void bm25_vocab_free(bm25_vocab* vocab);

/* ------------------------------------------------------ query-time scoring */

/* The paper's index stores S(t,D) for fixed k1, b (and delta); its
 * conclusion notes that Rank-BM25, which scores lazily, can change k1 at
 * inference.  These two calls give an index that: the postings are kept a
 * second time with TF and |D| in place of the score, and retrieval computes
 * S(t,D) - S0(t) from them with the call's k1, b, delta (same formulas,
 * same FP32 arithmetic per entry as the build, K_D in FP32), and adds
 * sum_i S0(q_i) at those parameters.  IDF does not depend on k1, b, delta
 * and is the index's.  With the index's own parameters the results equal
 * bm25_retrieve's up to FP32 rounding.
 *
 * bm25_index_enable_lazy builds the lazy postings (nnz + vocab + 3 pairs;
 * TF and |D| in 16 bits each when every TF and |D| fits, else TF in 32 bits
 * and |D| read from the document lengths).  Synchronous; idempotent.
 *
 * bm25_retrieve_lazy: arguments and results as bm25_retrieve, plus the
 * query-time k1 >= 0, 0 <= b <= 1, delta >= 0 (BM25L: k1 + delta > 0;
 * TFLDP: delta > 1/e).  Every query takes the doc-tiled path.  Uses the
 * index's default workspace.  BM25_E_INVALID without enable_lazy. */
int bm25_index_enable_lazy(bm25_index* index, void* cuda_stream);
int bm25_retrieve_lazy(const bm25_index* index, const int32_t* query_tokens,
                       int64_t n_query_tokens, const int64_t* query_offsets, int32_t n_queries,
                       int32_t k, double k1, double b, double delta, int32_t* out_ids,
                       float* out_scores, void* cuda_stream);

/* ------------------------------------------------------- doc-range shards */

/* A collection too large for one index is split into contiguous document
 * ranges, one index per range (one per GPU; the paper's Sec. 2.1 footnote
 * puts a dense 2M x 200K matrix at 1.6 TB, and the sparse one grows with the
 * collection too).  Every score must still use the WHOLE collection's DF, N
 * and Lavg, so building a shard takes two steps around one exchange:
 *   1. bm25_index_build over the range's documents (local ids 0 .. n-1);
 *      bm25_index_df_device gives its DF, bm25_index_info its N and tokens;
 *   2. the caller sums DF[vocab], N and the token count over the shards
 *      (an all-reduce), then bm25_index_rescore applies them.
 * A rescored shard's stored scores, IDF, S0 and Lavg equal those of one
 * index over the whole collection bit for bit (same arithmetic, same
 * inputs), and its retrieval returns global doc ids (local + doc_id_offset).
 * A query's top k over the collection is then the merge of every shard's
 * top k (an all-gather of the rows, then bm25_merge_topk). */

/* Copies the index's DF (its column lengths, int32 [vocab]) to df_out
 * (device).  Asynchronous on cuda_stream. */
int bm25_index_df_device(const bm25_index* index, int32_t* df_out, void* cuda_stream);

/* Recomputes IDF, S0, Lavg and every stored score from the collection's
 * statistics: global_df[vocab] (device int32, the sum of every shard's DF;
 * NULL = this index's own), global_n_docs (N of the collection, >= this
 * index's n_docs) and global_n_tokens (>= its n_tokens); Lavg =
 * global_n_tokens / global_n_docs.  doc_id_offset: the global id of this
 * index's document 0 (doc_id_offset + n_docs <= global_n_docs), added to
 * every id retrieval returns.  The structure (TF, DF, |D|, indptr, indices)
 * is unchanged.  Stream-ordered on cuda_stream; no retrieval on the index
 * may run meanwhile. */
int bm25_index_rescore(bm25_index* index, const int32_t* global_df, int64_t global_n_docs,
                       int64_t global_n_tokens, int64_t doc_id_offset, void* cuda_stream);

/* The shard parameters of an index (0, its own N and tokens unless
 * rescored).  Any pointer may be NULL.  Host memory. */
int bm25_index_shard_info(const bm25_index* index, int64_t* doc_id_offset,
                          int64_t* global_n_docs, int64_t* global_n_tokens);

/* Merges the top-k rows of n_shards shards: cand_ids / cand_scores are
 * [n_shards][n_queries][k] (device; id -1 marks an empty slot, as the
 * retrieval of a shard with fewer than k documents leaves them).  Row q of
 * out_ids / out_scores ([n_queries][k], device) gets the min(k, valid slots)
 * best by score descending, doc id ascending among equal scores, then -1 /
 * -inf.  1 <= k <= BM25_MAX_K.  Asynchronous on cuda_stream. */
int bm25_merge_topk(const int32_t* cand_ids, const float* cand_scores, int32_t n_shards,
                    int32_t n_queries, int32_t k, int32_t* out_ids, float* out_scores,
                    void* cuda_stream);

/* ---------------------------------------------------------------- serving */

/* A request loop over resident indexes with continuous batching (the paper
 * has no serving layer; this is the batched path of Sec. 2 run as requests
 * arrive).  Each request is one query (HOST tokens) against one index with
 * its own k.  A worker thread keeps up to max_inflight batches on the device
 * at once, each on its own stream and workspace; whenever one completes, the
 * requests that arrived meanwhile are batched per index (oldest first, up to
 * max_batch_queries) and admitted if the scratch of all running batches
 * stays within memory_budget (else a smaller batch, or after a running batch
 * completes).  A request's result does not depend on the batch it ran in
 * beyond the order of FP32 additions.  Each index's plan is used as set
 * (bm25_index_set_plan / bm25_autotune); the indexes must outlive the server
 * and must not be freed or re-planned while it runs. */
typedef struct bm25_server bm25_server;

typedef struct bm25_server_config {  /* zero fields take the defaults */
    int32_t max_batch_queries;  /* queries per batch (2048) */
    int32_t max_inflight;       /* batches on the device at once, <= 16 (3) */
    int32_t k_max;              /* largest k a request may ask for, <= BM25_MAX_K (1000) */
    int32_t reserved;           /* 0 */
    int64_t memory_budget;      /* device scratch bytes all batches may hold (4 GiB) */
} bm25_server_config;

typedef struct bm25_server_stats {
    int64_t completed, failed;  /* requests */
    int64_t batches, batched_queries;
    double p50_us, p99_us, max_us;  /* submit-to-result latency of completed requests */
    int64_t bytes_held;         /* device scratch the server holds now */
    double span_us;             /* first submit to last completion (the results ready on the
                                   host), so that completed / span is the served rate */
} bm25_server_stats;

/* Starts the worker thread.  indexes[n_indexes] live on the current device;
 * request index ids are positions in this array.  cfg may be NULL. */
int bm25_server_create(const bm25_index* const* indexes, int32_t n_indexes,
                       const bm25_server_config* cfg, bm25_server** out);

/* Queues one query: tokens[n_tokens] in HOST memory (copied; n_tokens may be
 * 0), checked against the index's vocabulary here (BM25_E_TOKEN_RANGE), and
 * 1 <= k <= k_max.  *ticket identifies the request in bm25_server_poll. */
int bm25_server_submit(bm25_server* server, int32_t index_id, const int32_t* tokens,
                       int32_t n_tokens, int32_t k, int64_t* ticket);

/* Waits up to timeout_us microseconds (0: do not wait, < 0: no limit) for a
 * request.  BM25_PENDING: not finished (poll again).  BM25_OK: ids[k] and
 * scores[k] (HOST, may be NULL) hold its row as bm25_retrieve would return
 * it, and the ticket is released.  A failed request returns its error code
 * once and releases the ticket. */
int bm25_server_poll(bm25_server* server, int64_t ticket, int32_t* ids, float* scores,
                     int32_t timeout_us);

/* Load replay, for measuring a server against the plain path under one
 * arrival process (the paper has no serving layer).  Request i asks index
 * index_ids[i] for its top ks[i] of the query tokens[offsets[i] ..
 * offsets[i+1]) (HOST arrays) and arrives arrival_s[i] seconds after the
 * call starts (non-decreasing).
 *
 * bm25_server_replay submits each request at its arrival time from the
 * calling thread and returns after the last submit; tickets[n] (HOST) get
 * the tickets (poll them as usual; the server's statistics time each request
 * from its submit).
 *
 * bm25_replay_plain answers the same requests one at a time, in order, each
 * by its own bm25_retrieve_host call (one query per call: copies in, the
 * launches, copies out, synchronise) on cuda_stream, starting each at its
 * arrival time or when the previous one is done; latency_us[n] (HOST) gets
 * each request's time from its arrival to its result. */
int bm25_server_replay(bm25_server* server, int32_t n, const int32_t* index_ids,
                       const int32_t* tokens, const int64_t* offsets, const int32_t* ks,
                       const double* arrival_s, int64_t* tickets);
int bm25_replay_plain(const bm25_index* const* indexes, int32_t n_indexes, int32_t n,
                      const int32_t* index_ids, const int32_t* tokens, const int64_t* offsets,
                      const int32_t* ks, const double* arrival_s, double* latency_us,
                      void* cuda_stream);

/* Counters and latency percentiles since the last reset (reset != 0 clears them). */
int bm25_server_stats_get(bm25_server* server, int reset, bm25_server_stats* out);

/* Stops accepting requests, lets running batches finish, fails queued
 * requests, joins the worker and frees the server's device memory. */
void bm25_server_destroy(bm25_server* server);

/* --------------------------------------------------------------- utility */

/* Message for the last failure on the calling thread ("" if none). */
const char* bm25_last_error(void);

/* Total number of kernels this library has launched in this process. */
int64_t bm25_launch_count(void);

/* Library version string. */
const char* bm25_version(void);

/* Per-kernel timing.  Between bm25_profile_begin() and bm25_profile_end()
 * every kernel launch of this library is bracketed by two CUDA events on the
 * stream it is launched on (not while that stream is being captured).
 * bm25_profile_end() waits for the recorded events and aggregates them per
 * kernel name; bm25_profile_count() and bm25_profile_get() read the result
 * (entry i: NUL-terminated name truncated to name_cap bytes, launch count,
 * summed milliseconds).  Off by default. */
int bm25_profile_begin(void);
int bm25_profile_end(void);
int bm25_profile_count(void);
int bm25_profile_get(int i, char* name, int name_cap, int64_t* launches, double* total_ms);

/* ------------------------------------------------------------ test hooks */

/* Failure injection for tests of the error paths (the paper has no
 * counterpart).  Both settings are process-wide and apply to every device.
 *
 * bm25_debug_set_handshake_polls: the number of polls after which a
 * producer/consumer wait of the doc-tiled retrieval kernel gives up
 * (default 2^22; polls < 0 restores it; 0 makes every such wait give up at
 * once).  A kernel that gives up records BM25_E_TIMEOUT in the index's
 * status word (read and cleared by bm25_sync_status), leaves its rows
 * undefined, waits for its own copies in flight and returns; the index and
 * the workspace stay usable.
 *
 * bm25_debug_fail_allocs: the next n device allocations the library makes
 * (index arrays, build scratch, workspace growth, host-path staging) fail
 * with BM25_E_OOM as if the device were out of memory (n <= 0 cancels). */
int bm25_debug_set_handshake_polls(int32_t polls);
int bm25_debug_fail_allocs(int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* BM25_GPU_H */
