// Internal declarations shared by the libbm25gpu translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "bm25.h"

namespace bm25 {

// ---- errors -----------------------------------------------------------
int set_error(int code, const char* fmt, ...);
void clear_error();

#define BM25_CUDA_TRY(expr)                                                         \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return ::bm25::set_error(e_ == cudaErrorMemoryAllocation ? BM25_E_OOM   \
                                                                     : BM25_E_CUDA, \
                                     "%s failed: %s (%s:%d)", #expr,                \
                                     cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

#define BM25_LAUNCH_CHECK() BM25_CUDA_TRY(cudaGetLastError())

#define BM25_TRY(expr)          \
    do {                        \
        int r_ = (expr);        \
        if (r_ != BM25_OK)      \
            return r_;          \
    } while (0)

// Test hooks (bm25_debug_*).  handshake_polls(): the poll limit of the tile
// kernel's producer/consumer waits (kHandshakePolls unless a test lowered
// it).  forced_alloc_failure(): true when a test asked for this device
// allocation to fail (consumes one of the failures it asked for).
constexpr int kHandshakePolls = 1 << 22;
int handshake_polls();
bool forced_alloc_failure();

// Kernel launch accounting (bm25_launch_count).
extern std::atomic<int64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Brackets one kernel launch with CUDA events while bm25_profile_begin() is
// active (no-op otherwise, and while the stream is being captured).
class ProfileScope {
public:
    ProfileScope(const char* name, cudaStream_t s);
    ~ProfileScope();
    ProfileScope(const ProfileScope&) = delete;
    ProfileScope& operator=(const ProfileScope&) = delete;

private:
    const char* name_;
    cudaStream_t s_;
    void* a_ = nullptr;
};

// Device properties of the current device, cached.
struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    int max_smem_optin = 0;
    int l2_bytes = 0;
};
int device_info(DeviceInfo* out);

// ---- the index --------------------------------------------------------
// Packed posting layout (bm25_index::posts): the first slot of column t.
// Rounding indptr[t] + t up to an even number keeps the columns disjoint
// (each gains at most one slot over the previous) and 16-byte aligned.
__host__ __device__ inline int64_t post_start(int64_t indptr_t, int64_t t)
{
    return (indptr_t + t + 1) & ~int64_t(1);
}
constexpr uint32_t kPostPad = 0xffffffffu;  // doc id of a padding slot (beyond any document)

struct Plan {
    int accumulator = BM25_ACC_AUTO;
    int32_t tile_docs = 6144;
    int32_t threads = 256;
    int32_t dense_max = 4096;   // postings bound of the dense path (AUTO, L2_DENSE)
    int32_t stage_entries = 1536; // packed postings per staging buffer of the tiled kernel
    int32_t stages = 2;           // staging buffers in its ring
};
// Fills zero fields of `in` from `base`; BM25_E_INVALID (nothing changed) if
// a field is out of range.
int merge_plan(const bm25_plan* in, const Plan& base, Plan* out);

}  // namespace bm25

struct bm25_index {
    int device = 0;
    int64_t n_docs = 0, n_tokens = 0, nnz = 0;
    int32_t vocab = 0;
    int variant = 0;
    double k1 = 0, b = 0, delta = 0, lavg = 0;
    // device arrays (owned)
    int64_t* indptr = nullptr;   // [vocab+1]
    int32_t* indices = nullptr;  // [nnz]   doc ids, ascending per term
    float* data = nullptr;       // [nnz]   S(t,D) - S0(t), FP32
    int32_t* tf = nullptr;       // [nnz]
    int32_t* df = nullptr;       // [vocab]
    int32_t* doc_len = nullptr;  // [n_docs]
    double* idf = nullptr;       // [vocab]
    double* s0 = nullptr;        // [vocab]
    // The same entries packed as (doc id, S - S0 bits) pairs for staged
    // retrieval: column t starts at post_start(indptr[t], t), an even
    // position, so every column begins on a 16-byte boundary; the 0-2 slots
    // between columns and the slots past the last one hold kPostPad.
    uint2* posts = nullptr;      // [n_posts]
    int64_t n_posts = 0;         // nnz + vocab + 3
    int* status = nullptr;       // device status word (first error code)
    // doc-range sharding: returned doc ids are local ids + doc_offset; IDF,
    // S0 and Lavg come from a collection of stat_docs documents and
    // stat_tokens tokens (this index's own counts unless rescored)
    int64_t doc_offset = 0;
    int64_t stat_docs = 0, stat_tokens = 0;
    // query-time scoring (bm25_index_enable_lazy): the packed layout again,
    // second word TF | |D| << 16 (lazy_packed) or TF alone
    uint2* posts_lazy = nullptr;  // [n_posts]
    bool lazy_packed = false;
    bm25::Plan plan;
    bm25_workspace* default_ws = nullptr;
    std::mutex mu;
};

struct bm25_workspace {
    int device = 0;
    bool fixed = false;  // buffers lent by the caller: never grown, never freed
    // per-query arrays, carved from qbuf (see bm25::carve_queries)
    unsigned char* qbuf = nullptr;
    size_t qbuf_cap = 0;             // bytes
    int32_t max_queries = 0;         // queries per sub-batch the arrays hold
    uint32_t* ctr = nullptr;         // [4] tiled count, dense count, dense queue head
    double* shift = nullptr;         // [q]  sum_i S0(q_i)
    int4* lrec = nullptr;            // [li] tiled-path record {q, first token, end token, k' and a flag}
    int32_t* qkp = nullptr;          // [q]  k' = min(k_q, N)
    uint32_t* lpost = nullptr;       // [li] postings of the query's columns
    uint32_t* thresh = nullptr;      // [li] running k'-th best score key
    int32_t* sq = nullptr;           // [si] dense-path queries
    // tiled path
    int32_t* seg = nullptr;          // [n_query_tokens * (n_tiles + 1)]
    uint32_t* tcount = nullptr;      // [n_tiles * queries]  candidates per (tile, query) item
    unsigned long long* cand = nullptr;  // [n_tiles * queries * kstride]
    size_t seg_cap = 0, cand_cap = 0, tcount_cap = 0;  // element capacities
    // dense path: one N-vector (all -0.0 between queries) and one candidate
    // list per CTA
    float* dslots = nullptr;
    unsigned long long* dlists = nullptr;
    size_t dslots_cap = 0, dlists_cap = 0;  // element capacities
    // staging for the _host entry points
    int32_t* q_tokens = nullptr;
    int64_t* q_offsets = nullptr;
    int32_t* q_k = nullptr;
    int32_t* out_ids = nullptr;
    float* out_scores = nullptr;
    size_t staging_cap[5] = {0, 0, 0, 0, 0};  // bytes
    bool owns_staging = false;
};

namespace bm25 {

// ---- build (index_build.cu) --------------------------------------------
int build_index_device(const int32_t* d_tokens, int64_t n_tokens, const int64_t* d_offsets,
                       int64_t n_docs, int32_t vocab, int variant, double k1, double b,
                       double delta, cudaStream_t stream, bm25_index** out);
// Allocates the index's V/N-sized arrays (fixed) and/or its nnz-sized arrays
// (per_entry) from the library's pool on stream s.
int alloc_index_arrays(bm25_index* ix, cudaStream_t s, bool fixed, bool per_entry);
void free_index_arrays(bm25_index* ix, cudaStream_t s);
// Fills ix->posts from indptr / indices / data (used after an import; the
// build writes the packed entries as it scores them).  Stream-ordered.
int pack_posts(bm25_index* ix, cudaStream_t s);
int rescore_index(bm25_index* ix, const int32_t* df_global, int64_t n_docs_global,
                  int64_t n_tokens_global, cudaStream_t s);
// Builds ix->posts_lazy from the CSC, TF and |D| (synchronous).
int enable_lazy(bm25_index* ix, cudaStream_t s);
int pool_for_current_device(cudaMemPool_t* out);

// ---- retrieval (retrieve.cu) -------------------------------------------
// Host-side checks of a retrieval call (api.cu): index, batch sizes, k and
// BM25_MAX_K, the current device.
int check_retrieve_args(const bm25_index* ix, int64_t n_tok, int32_t nq, int32_t k);
// Query-time parameters of lazy scoring (bm25_retrieve_lazy).
struct QueryParams {
    double k1, b, delta;
};
// q_k: per-query k (device, NULL = k_max for every query); rows of the
// outputs are k_max wide.  qp: score at query time with these parameters
// from the index's lazy postings (every query on the doc-tiled path), or
// NULL for the stored scores.
int retrieve_device(const bm25_index* ix, bm25_workspace* ws, const int32_t* q_tokens,
                    const int64_t* q_offsets, int32_t n_queries, int64_t n_query_tokens,
                    const int32_t* q_k, int32_t k_max, int32_t* out_ids, float* out_scores,
                    const Plan& plan, cudaStream_t stream, const QueryParams* qp = nullptr);
// Grows ws (unless fixed) to what retrieve_device needs for such a call;
// allocates nothing when it already fits.  Fails while `stream` is being
// captured and something would have to grow.
int workspace_reserve_for(const bm25_index* ix, bm25_workspace* ws, int32_t n_queries,
                          int64_t n_query_tokens, int32_t k_max, const Plan& plan,
                          cudaStream_t stream);
void workspace_release(bm25_workspace* ws);
// Merge of n_shards top-k rows per query ([n_shards][n_queries][k] device
// arrays, ids -1 for empty slots) into [n_queries][k] by (score desc, id asc).
int merge_topk_device(const int32_t* cand_ids, const float* cand_scores, int32_t n_shards,
                      int32_t n_queries, int32_t k, int32_t* out_ids, float* out_scores,
                      cudaStream_t s);
// Device bytes a workspace needs for such a call (from scratch), and the
// bytes a workspace holds now.
int workspace_bytes_for(const bm25_index* ix, int32_t n_queries, int64_t n_query_tokens,
                        int32_t k_max, const Plan& plan, size_t* bytes);
size_t workspace_bytes_held(const bm25_workspace* ws);
// Bytes of the per-query arrays for m queries, and their carve-up of qbuf.
size_t query_arrays_bytes(int64_t m);
void carve_queries(bm25_workspace* ws, unsigned char* base, int32_t m);
// The doc-tile width a plan gives for an index of n_docs documents.
int32_t tile_width(const Plan& plan, int64_t n_docs);

// ---- scan (scan.cu) ------------------------------------------------------
// Exclusive prefix sum of n uint32 values (in and out may alias).  The total
// goes to d_total (device).  tmp needs scan_tmp_elems(n) uint32 of scratch.
int64_t scan_tmp_elems(int64_t n);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                       uint32_t* tmp, cudaStream_t stream);

}  // namespace bm25
