// The C ABI of libbm25gpu (declared in include/bm25.h): argument checks,
// host-buffer variants, checkpoint export/import, status and error reporting.
// All compute is in index_build.cu, retrieve.cu and scan.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace bm25 {

std::atomic<int64_t> g_launches{0};

namespace {
thread_local char g_err[1024] = {0};

std::mutex g_dev_mu;
DeviceInfo g_dev[64];
}  // namespace

int set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

namespace {
std::atomic<int> g_handshake_polls{kHandshakePolls};
std::atomic<int> g_fail_allocs{0};
}  // namespace

int handshake_polls() { return g_handshake_polls.load(std::memory_order_relaxed); }

bool forced_alloc_failure()
{
    int n = g_fail_allocs.load(std::memory_order_relaxed);
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1, std::memory_order_relaxed))
            return true;
    }
    return false;
}

int device_info(DeviceInfo* out)
{
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return set_error(BM25_E_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (g_dev[dev].device != dev) {
        DeviceInfo d;
        d.device = dev;
        BM25_CUDA_TRY(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
        BM25_CUDA_TRY(cudaDeviceGetAttribute(&d.max_smem_optin,
                                             cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        BM25_CUDA_TRY(cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev));
        g_dev[dev] = d;
    }
    *out = g_dev[dev];
    return BM25_OK;
}

// Host-side checks shared by every retrieval entry point.
int check_retrieve_args(const bm25_index* ix, int64_t n_tok, int32_t nq, int32_t k)
{
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    if (nq < 0 || n_tok < 0 || n_tok > (int64_t)INT32_MAX)
        return set_error(BM25_E_INVALID, "bad batch size (n_queries %d, n_query_tokens %lld)", nq,
                         (long long)n_tok);
    if (k < 1)
        return set_error(BM25_E_INVALID, "k = %d must be >= 1", k);
    int64_t kp = k < ix->n_docs ? k : ix->n_docs;
    if (kp > BM25_MAX_K)
        return set_error(BM25_E_INVALID, "min(k, n_docs) = %lld exceeds BM25_MAX_K = %d",
                         (long long)kp, BM25_MAX_K);
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ix->device)
        return set_error(BM25_E_INVALID, "current device %d is not the index's device %d", dev,
                         ix->device);
    return BM25_OK;
}

namespace {

int check_build_args(int64_t n_tokens, int64_t n_docs, int32_t vocab, int variant, double k1,
                     double b, double delta, bm25_index** out)
{
    if (!out)
        return set_error(BM25_E_INVALID, "out is NULL");
    *out = nullptr;
    if (variant < BM25_LUCENE || variant > BM25_TFLDP)
        return set_error(BM25_E_INVALID, "unknown variant %d", variant);
    if (n_docs < 1 || n_docs > (int64_t)INT32_MAX - 1)
        return set_error(BM25_E_INVALID, "n_docs = %lld outside [1, 2^31 - 2]", (long long)n_docs);
    if (n_tokens < 0 || n_tokens > (int64_t)INT32_MAX - 1)
        return set_error(BM25_E_INVALID, "n_tokens = %lld outside [0, 2^31 - 2]",
                         (long long)n_tokens);
    if (vocab < 1 || vocab == INT32_MAX)
        return set_error(BM25_E_INVALID, "vocab = %d must be in [1, 2^31 - 2]", vocab);
    if (!(k1 >= 0.0) || !(b >= 0.0 && b <= 1.0) || !(delta >= 0.0))
        return set_error(BM25_E_INVALID, "need k1 >= 0, 0 <= b <= 1, delta >= 0 (got %g, %g, %g)",
                         k1, b, delta);
    if (variant == BM25_L && !(k1 + delta > 0.0))
        return set_error(BM25_E_INVALID, "BM25L needs k1 + delta > 0");
    if (variant == BM25_TFLDP && !(1.0 + log(delta) > 0.0))
        return set_error(BM25_E_INVALID, "TFLDP needs delta > 1/e (got %g)", delta);
    return BM25_OK;
}

Plan plan_of(const bm25_index* ix)
{
    std::lock_guard<std::mutex> g(const_cast<bm25_index*>(ix)->mu);
    return ix->plan;
}

// The default workspace of a freed index is kept (one per device) and handed
// to the next index's first call, so that building and dropping indexes in a
// loop allocates retrieval scratch once.  Its buffers grow on demand and the
// dense-path vectors are left at -0.0 by every query, so nothing carries over.
std::mutex g_ws_cache_mu;
bm25_workspace* g_ws_cache[64] = {};

bm25_workspace* take_cached_ws(int dev)
{
    std::lock_guard<std::mutex> g(g_ws_cache_mu);
    if (dev < 0 || dev >= 64)
        return nullptr;
    bm25_workspace* ws = g_ws_cache[dev];
    g_ws_cache[dev] = nullptr;
    return ws;
}

void put_cached_ws(bm25_workspace* ws)
{
    {
        std::lock_guard<std::mutex> g(g_ws_cache_mu);
        if (ws->device >= 0 && ws->device < 64 && !g_ws_cache[ws->device]) {
            g_ws_cache[ws->device] = ws;
            return;
        }
    }
    workspace_release(ws);
    delete ws;
}

int default_ws(const bm25_index* ix, bm25_workspace** out)
{
    bm25_index* m = const_cast<bm25_index*>(ix);
    if (!m->default_ws) {
        bm25_workspace* ws = take_cached_ws(ix->device);
        if (!ws) {
            ws = new bm25_workspace();
            ws->device = ix->device;
        }
        m->default_ws = ws;
    }
    *out = m->default_ws;
    return BM25_OK;
}

}  // namespace

int merge_plan(const bm25_plan* in, const Plan& base, Plan* out)
{
    Plan p = base;
    if (in) {
        if (in->dense_max_postings < 0 || in->dense_max_postings > (1 << 22))
            return set_error(BM25_E_INVALID, "dense_max_postings %d must be in [0, 2^22]",
                             in->dense_max_postings);
        if (in->accumulator < BM25_ACC_UNSET || in->accumulator > BM25_ACC_L2_DENSE)
            return set_error(BM25_E_INVALID, "unknown accumulator %d", in->accumulator);
        if (in->tile_docs != 0 &&
            (in->tile_docs < 1024 || in->tile_docs > 49152 || in->tile_docs % 1024))
            return set_error(BM25_E_INVALID,
                             "tile_docs %d must be a multiple of 1024 in [1024, 49152]",
                             in->tile_docs);
        if (in->block_threads != 0 && in->block_threads != 128 && in->block_threads != 192 &&
            in->block_threads != 256 && in->block_threads != 512)
            return set_error(BM25_E_INVALID, "block_threads %d must be 128, 192, 256 or 512",
                             in->block_threads);
        if (in->stage_entries != 0 &&
            (in->stage_entries < 128 || in->stage_entries > 8192 || in->stage_entries % 64))
            return set_error(BM25_E_INVALID,
                             "stage_entries %d must be a multiple of 64 in [128, 8192]",
                             in->stage_entries);
        if (in->stages != 0 && (in->stages < 2 || in->stages > 8))
            return set_error(BM25_E_INVALID, "stages %d must be in [2, 8]", in->stages);
        if (in->stage_entries)
            p.stage_entries = in->stage_entries;
        if (in->stages)
            p.stages = in->stages;
        if (in->accumulator)
            p.accumulator = in->accumulator;
        if (in->tile_docs)
            p.tile_docs = in->tile_docs;
        if (in->block_threads)
            p.threads = in->block_threads;
        if (in->dense_max_postings)
            p.dense_max = in->dense_max_postings;
    }
    *out = p;
    return BM25_OK;
}

}  // namespace bm25

using namespace bm25;

extern "C" {

const char* bm25_last_error(void) { return g_err; }

int64_t bm25_launch_count(void) { return g_launches.load(); }

const char* bm25_version(void) { return "bm25gpu 0.1 (sm_103a)"; }

int bm25_index_build(const int32_t* token_ids, int64_t n_tokens, const int64_t* doc_offsets,
                     int64_t n_docs, int32_t vocab, int variant, double k1, double b, double delta,
                     void* cuda_stream, bm25_index** out)
{
    clear_error();
    BM25_TRY(check_build_args(n_tokens, n_docs, vocab, variant, k1, b, delta, out));
    if (!doc_offsets || (n_tokens > 0 && !token_ids))
        return set_error(BM25_E_INVALID, "NULL input array");
    return build_index_device(token_ids, n_tokens, doc_offsets, n_docs, vocab, variant, k1, b,
                              delta, (cudaStream_t)cuda_stream, out);
}

int bm25_index_build_host(const int32_t* token_ids, int64_t n_tokens, const int64_t* doc_offsets,
                          int64_t n_docs, int32_t vocab, int variant, double k1, double b,
                          double delta, void* cuda_stream, bm25_index** out)
{
    clear_error();
    BM25_TRY(check_build_args(n_tokens, n_docs, vocab, variant, k1, b, delta, out));
    if (!doc_offsets || (n_tokens > 0 && !token_ids))
        return set_error(BM25_E_INVALID, "NULL input array");
    if (doc_offsets[0] != 0 || doc_offsets[n_docs] != n_tokens)
        return set_error(BM25_E_INVALID, "doc_offsets must start at 0 and end at n_tokens");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaMemPool_t pool;
    BM25_TRY(pool_for_current_device(&pool));
    int32_t* d_tok = nullptr;
    int64_t* d_off = nullptr;
    BM25_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_tok, sizeof(int32_t) * (n_tokens + 1), pool, s));
    cudaError_t e = cudaMallocFromPoolAsync((void**)&d_off, sizeof(int64_t) * (n_docs + 1), pool, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(d_tok, s);
        return set_error(BM25_E_OOM, "device allocation failed: %s", cudaGetErrorString(e));
    }
    int rc = BM25_OK;
    if (n_tokens > 0 && cudaMemcpyAsync(d_tok, token_ids, sizeof(int32_t) * n_tokens,
                                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "token copy failed");
    if (rc == BM25_OK && cudaMemcpyAsync(d_off, doc_offsets, sizeof(int64_t) * (n_docs + 1),
                                         cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "offset copy failed");
    if (rc == BM25_OK)
        rc = build_index_device(d_tok, n_tokens, d_off, n_docs, vocab, variant, k1, b, delta, s,
                                out);
    cudaFreeAsync(d_tok, s);
    cudaFreeAsync(d_off, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == BM25_OK)
        rc = set_error(BM25_E_CUDA, "stream synchronisation failed");
    return rc;
}

int bm25_index_info(const bm25_index* ix, int64_t* n_docs, int64_t* n_tokens, int64_t* nnz,
                    int32_t* vocab, int* variant, double* k1, double* b, double* delta,
                    double* lavg)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    if (n_docs) *n_docs = ix->n_docs;
    if (n_tokens) *n_tokens = ix->n_tokens;
    if (nnz) *nnz = ix->nnz;
    if (vocab) *vocab = ix->vocab;
    if (variant) *variant = ix->variant;
    if (k1) *k1 = ix->k1;
    if (b) *b = ix->b;
    if (delta) *delta = ix->delta;
    if (lavg) *lavg = ix->lavg;
    return BM25_OK;
}

int bm25_index_export(const bm25_index* ix, int64_t* indptr, int32_t* indices, float* data,
                      int32_t* tf, int32_t* df, int32_t* doc_len, double* idf, double* s0)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    BM25_CUDA_TRY(cudaDeviceSynchronize());
    auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
        if (dst && bytes)
            BM25_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        return BM25_OK;
    };
    BM25_TRY(cp(indptr, ix->indptr, sizeof(int64_t) * (ix->vocab + 1)));
    BM25_TRY(cp(indices, ix->indices, sizeof(int32_t) * ix->nnz));
    BM25_TRY(cp(data, ix->data, sizeof(float) * ix->nnz));
    BM25_TRY(cp(tf, ix->tf, sizeof(int32_t) * ix->nnz));
    BM25_TRY(cp(df, ix->df, sizeof(int32_t) * ix->vocab));
    BM25_TRY(cp(doc_len, ix->doc_len, sizeof(int32_t) * ix->n_docs));
    BM25_TRY(cp(idf, ix->idf, sizeof(double) * ix->vocab));
    BM25_TRY(cp(s0, ix->s0, sizeof(double) * ix->vocab));
    return BM25_OK;
}

int bm25_index_import(int64_t n_docs, int64_t n_tokens, int64_t nnz, int32_t vocab, int variant,
                      double k1, double b, double delta, double lavg, const int64_t* indptr,
                      const int32_t* indices, const float* data, const int32_t* tf,
                      const int32_t* df, const int32_t* doc_len, const double* idf,
                      const double* s0, bm25_index** out)
{
    clear_error();
    BM25_TRY(check_build_args(n_tokens, n_docs, vocab, variant, k1, b, delta, out));
    if (nnz < 0 || nnz > n_tokens || !indptr || !df || !doc_len || !idf || !s0 ||
        (nnz > 0 && (!indices || !data)))
        return set_error(BM25_E_INVALID, "bad import arrays");
    // structure checks: the retrieval kernels rely on them
    if (indptr[0] != 0 || indptr[vocab] != nnz)
        return set_error(BM25_E_INVALID, "indptr must run from 0 to nnz");
    for (int32_t t = 0; t < vocab; t++) {
        if (indptr[t + 1] < indptr[t])
            return set_error(BM25_E_INVALID, "indptr decreases at term %d", t);
        for (int64_t j = indptr[t]; j < indptr[t + 1]; j++) {
            if (indices[j] < 0 || indices[j] >= n_docs ||
                (j > indptr[t] && indices[j] <= indices[j - 1]))
                return set_error(BM25_E_INVALID, "column %d is not strictly ascending in [0, N)", t);
        }
    }
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    bm25_index* ix = new bm25_index();
    ix->device = dev;
    ix->n_docs = n_docs;
    ix->n_tokens = n_tokens;
    ix->nnz = nnz;
    ix->vocab = vocab;
    ix->variant = variant;
    ix->k1 = k1;
    ix->b = b;
    ix->delta = delta;
    ix->lavg = lavg;
    ix->stat_docs = n_docs;
    ix->stat_tokens = n_tokens;
    int rc = alloc_index_arrays(ix, 0, true, true);
    auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
        if (bytes)
            BM25_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return BM25_OK;
    };
    if (rc == BM25_OK) rc = cp(ix->indptr, indptr, sizeof(int64_t) * (vocab + 1));
    if (rc == BM25_OK) rc = cp(ix->indices, indices, sizeof(int32_t) * nnz);
    if (rc == BM25_OK && nnz > 0) {
        // stored scores never hold -0.0 (retrieval marks untouched documents with it)
        std::vector<float> d(data, data + nnz);
        for (float& x : d)
            if (x == 0.0f)
                x = 0.0f;
        rc = cp(ix->data, d.data(), sizeof(float) * nnz);
    }
    if (rc == BM25_OK) {
        if (tf)
            rc = cp(ix->tf, tf, sizeof(int32_t) * nnz);
        else if (nnz && cudaMemset(ix->tf, 0, sizeof(int32_t) * nnz) != cudaSuccess)
            rc = set_error(BM25_E_CUDA, "memset failed");
    }
    if (rc == BM25_OK) rc = cp(ix->df, df, sizeof(int32_t) * vocab);
    if (rc == BM25_OK) rc = cp(ix->doc_len, doc_len, sizeof(int32_t) * n_docs);
    if (rc == BM25_OK) rc = cp(ix->idf, idf, sizeof(double) * vocab);
    if (rc == BM25_OK) rc = cp(ix->s0, s0, sizeof(double) * vocab);
    if (rc == BM25_OK) rc = pack_posts(ix, 0);
    if (rc == BM25_OK && cudaDeviceSynchronize() != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "synchronisation failed");
    if (rc != BM25_OK) {
        free_index_arrays(ix, 0);
        delete ix;
        return rc;
    }
    *out = ix;
    return BM25_OK;
}

int bm25_sync_status(const bm25_index* ix, void* cuda_stream)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int h = 0;
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    BM25_CUDA_TRY(cudaMemcpy(&h, ix->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        BM25_CUDA_TRY(cudaMemset(ix->status, 0, sizeof(int)));
        return set_error(h, "a kernel recorded error %d (token id outside [0, vocab) or "
                            "malformed offsets)", h);
    }
    return BM25_OK;
}

void bm25_index_free(bm25_index* ix)
{
    if (!ix)
        return;
    if (ix->default_ws)
        put_cached_ws(ix->default_ws);
    free_index_arrays(ix, 0);
    cudaStreamSynchronize(0);
    delete ix;
}

void bm25_release_cached(void)
{
    for (int d = 0; d < 64; d++) {
        bm25_workspace* ws = take_cached_ws(d);
        if (!ws)
            continue;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(d);
        workspace_release(ws);
        delete ws;
        cudaSetDevice(cur);
    }
}

int bm25_workspace_create(const bm25_index* ix, int32_t max_queries, int64_t max_query_tokens,
                          int32_t max_k, bm25_workspace** out)
{
    clear_error();
    if (!out || !ix)
        return set_error(BM25_E_INVALID, "NULL argument");
    *out = nullptr;
    if (max_queries < 1 || max_query_tokens < 0 || max_k < 1)
        return set_error(BM25_E_INVALID, "bad workspace limits");
    BM25_TRY(check_retrieve_args(ix, max_query_tokens, max_queries, max_k));
    bm25_workspace* ws = new bm25_workspace();
    ws->device = ix->device;
    int rc = workspace_reserve_for(ix, ws, max_queries, max_query_tokens, max_k, plan_of(ix), 0);
    if (rc == BM25_OK && cudaStreamSynchronize(0) != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "synchronisation failed");
    if (rc != BM25_OK) {
        workspace_release(ws);
        delete ws;
        return rc;
    }
    *out = ws;
    return BM25_OK;
}

int bm25_workspace_reserve(bm25_workspace* ws, const bm25_index* ix, int32_t n_queries,
                           int64_t n_query_tokens, int32_t k_max, const bm25_plan* plan,
                           void* cuda_stream)
{
    clear_error();
    if (!ws)
        return set_error(BM25_E_INVALID, "workspace is NULL");
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k_max));
    if (ws->device != ix->device)
        return set_error(BM25_E_INVALID, "workspace and index are on different devices");
    Plan p;
    BM25_TRY(merge_plan(plan, plan_of(ix), &p));
    return workspace_reserve_for(ix, ws, n_queries, n_query_tokens, k_max, p,
                                 (cudaStream_t)cuda_stream);
}

void bm25_workspace_free(bm25_workspace* ws)
{
    if (!ws)
        return;
    workspace_release(ws);
    delete ws;
}

int bm25_retrieve(const bm25_index* ix, const int32_t* query_tokens, int64_t n_query_tokens,
                  const int64_t* query_offsets, int32_t n_queries, int32_t k, int32_t* out_ids,
                  float* out_scores, void* cuda_stream)
{
    clear_error();
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k));
    bm25_workspace* ws = nullptr;
    BM25_TRY(default_ws(ix, &ws));
    return retrieve_device(ix, ws, query_tokens, query_offsets, n_queries, n_query_tokens,
                           nullptr, k, out_ids, out_scores, plan_of(ix),
                           (cudaStream_t)cuda_stream);
}

int bm25_index_enable_lazy(bm25_index* ix, void* cuda_stream)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ix->device)
        return set_error(BM25_E_INVALID, "current device %d is not the index's device %d", dev,
                         ix->device);
    std::lock_guard<std::mutex> g(ix->mu);
    return enable_lazy(ix, (cudaStream_t)cuda_stream);
}

int bm25_retrieve_lazy(const bm25_index* ix, const int32_t* query_tokens, int64_t n_query_tokens,
                       const int64_t* query_offsets, int32_t n_queries, int32_t k, double k1,
                       double b, double delta, int32_t* out_ids, float* out_scores,
                       void* cuda_stream)
{
    clear_error();
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k));
    if (!ix->posts_lazy)
        return set_error(BM25_E_INVALID, "the index has no lazy postings: call "
                         "bm25_index_enable_lazy first");
    if (!(k1 >= 0.0) || !(b >= 0.0 && b <= 1.0) || !(delta >= 0.0))
        return set_error(BM25_E_INVALID, "need k1 >= 0, 0 <= b <= 1, delta >= 0 (got %g, %g, %g)",
                         k1, b, delta);
    if (ix->variant == BM25_L && !(k1 + delta > 0.0))
        return set_error(BM25_E_INVALID, "BM25L needs k1 + delta > 0");
    if (ix->variant == BM25_TFLDP && !(1.0 + log(delta) > 0.0))
        return set_error(BM25_E_INVALID, "TFLDP needs delta > 1/e (got %g)", delta);
    bm25_workspace* ws = nullptr;
    BM25_TRY(default_ws(ix, &ws));
    Plan p = plan_of(ix);
    p.accumulator = BM25_ACC_SMEM_TILED;
    const QueryParams qp{k1, b, delta};
    return retrieve_device(ix, ws, query_tokens, query_offsets, n_queries, n_query_tokens,
                           nullptr, k, out_ids, out_scores, p, (cudaStream_t)cuda_stream, &qp);
}

int bm25_retrieve_ws(const bm25_index* ix, bm25_workspace* ws, const int32_t* query_tokens,
                     int64_t n_query_tokens, const int64_t* query_offsets, int32_t n_queries,
                     int32_t k, int32_t* out_ids, float* out_scores, const bm25_plan* plan,
                     void* cuda_stream)
{
    clear_error();
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k));
    if (!ws)
        return set_error(BM25_E_INVALID, "workspace is NULL");
    Plan p;
    BM25_TRY(merge_plan(plan, plan_of(ix), &p));
    return retrieve_device(ix, ws, query_tokens, query_offsets, n_queries, n_query_tokens,
                           nullptr, k, out_ids, out_scores, p, (cudaStream_t)cuda_stream);
}

int bm25_retrieve_batch(const bm25_index* ix, bm25_workspace* ws, const int32_t* query_tokens,
                        int64_t n_query_tokens, const int64_t* query_offsets, int32_t n_queries,
                        const int32_t* query_k, int32_t k_max, int32_t* out_ids,
                        float* out_scores, const bm25_plan* plan, void* cuda_stream)
{
    clear_error();
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k_max));
    if (n_queries > 0 && (!query_offsets || !out_ids || !out_scores ||
                          (n_query_tokens > 0 && !query_tokens)))
        return set_error(BM25_E_INVALID, "NULL array");
    if (!ws)
        BM25_TRY(default_ws(ix, &ws));
    else if (ws->device != ix->device)
        return set_error(BM25_E_INVALID, "workspace and index are on different devices");
    Plan p;
    BM25_TRY(merge_plan(plan, plan_of(ix), &p));
    return retrieve_device(ix, ws, query_tokens, query_offsets, n_queries, n_query_tokens,
                           query_k, k_max, out_ids, out_scores, p, (cudaStream_t)cuda_stream);
}

int bm25_retrieve_host(const bm25_index* ix, const int32_t* query_tokens,
                       const int64_t* query_offsets, int32_t n_queries, int32_t k,
                       int32_t* out_ids, float* out_scores, void* cuda_stream)
{
    clear_error();
    if (!query_offsets || (n_queries > 0 && (!out_ids || !out_scores)))
        return set_error(BM25_E_INVALID, "NULL argument");
    if (n_queries < 0)
        return set_error(BM25_E_INVALID, "n_queries < 0");
    if (query_offsets[0] != 0)
        return set_error(BM25_E_INVALID, "query_offsets[0] must be 0");
    const int64_t n_tok = query_offsets[n_queries];
    BM25_TRY(check_retrieve_args(ix, n_tok, n_queries, k));
    if (n_queries == 0)
        return BM25_OK;
    bm25_workspace* ws = nullptr;
    BM25_TRY(default_ws(ix, &ws));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // staging buffers, grown as needed
    static_assert(sizeof(int32_t) == 4, "");
    auto grow = [&](void** p, size_t* cap, size_t bytes) -> int {
        if (*cap >= bytes && *p)
            return BM25_OK;
        if (*p)
            cudaFree(*p);
        *p = nullptr;
        *cap = 0;
        if (forced_alloc_failure())
            return set_error(BM25_E_OOM, "device allocation of %zu bytes failed (forced by "
                             "bm25_debug_fail_allocs)", bytes);
        BM25_CUDA_TRY(cudaMalloc(p, bytes ? bytes : 1));
        *cap = bytes;
        return BM25_OK;
    };
    ws->owns_staging = true;
    BM25_TRY(grow((void**)&ws->q_tokens, &ws->staging_cap[0], sizeof(int32_t) * (size_t)n_tok));
    BM25_TRY(grow((void**)&ws->q_offsets, &ws->staging_cap[1],
                  sizeof(int64_t) * (size_t)(n_queries + 1)));
    BM25_TRY(grow((void**)&ws->out_ids, &ws->staging_cap[3],
                  sizeof(int32_t) * (size_t)n_queries * k));
    BM25_TRY(grow((void**)&ws->out_scores, &ws->staging_cap[4],
                  sizeof(float) * (size_t)n_queries * k));
    if (n_tok > 0)
        BM25_CUDA_TRY(cudaMemcpyAsync(ws->q_tokens, query_tokens, sizeof(int32_t) * n_tok,
                                      cudaMemcpyHostToDevice, s));
    BM25_CUDA_TRY(cudaMemcpyAsync(ws->q_offsets, query_offsets,
                                  sizeof(int64_t) * (n_queries + 1), cudaMemcpyHostToDevice, s));
    BM25_TRY(retrieve_device(ix, ws, ws->q_tokens, ws->q_offsets, n_queries, n_tok, nullptr, k,
                             ws->out_ids, ws->out_scores, plan_of(ix), s));
    BM25_CUDA_TRY(cudaMemcpyAsync(out_ids, ws->out_ids, sizeof(int32_t) * (size_t)n_queries * k,
                                  cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaMemcpyAsync(out_scores, ws->out_scores,
                                  sizeof(float) * (size_t)n_queries * k, cudaMemcpyDeviceToHost,
                                  s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    return BM25_OK;
}

int bm25_index_df_device(const bm25_index* ix, int32_t* df_out, void* cuda_stream)
{
    clear_error();
    if (!ix || !df_out)
        return set_error(BM25_E_INVALID, "NULL argument");
    BM25_CUDA_TRY(cudaMemcpyAsync(df_out, ix->df, sizeof(int32_t) * (size_t)ix->vocab,
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)cuda_stream));
    return BM25_OK;
}

int bm25_index_rescore(bm25_index* ix, const int32_t* global_df, int64_t global_n_docs,
                       int64_t global_n_tokens, int64_t doc_id_offset, void* cuda_stream)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    if (global_n_docs < ix->n_docs || global_n_docs > (int64_t)INT32_MAX - 1)
        return set_error(BM25_E_INVALID, "global_n_docs %lld outside [n_docs %lld, 2^31 - 2]",
                         (long long)global_n_docs, (long long)ix->n_docs);
    if (global_n_tokens < ix->n_tokens)
        return set_error(BM25_E_INVALID, "global_n_tokens %lld is below the index's %lld",
                         (long long)global_n_tokens, (long long)ix->n_tokens);
    if (doc_id_offset < 0 || doc_id_offset + ix->n_docs > global_n_docs)
        return set_error(BM25_E_INVALID, "doc range [%lld, %lld) outside [0, %lld)",
                         (long long)doc_id_offset, (long long)(doc_id_offset + ix->n_docs),
                         (long long)global_n_docs);
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ix->device)
        return set_error(BM25_E_INVALID, "current device %d is not the index's device %d", dev,
                         ix->device);
    std::lock_guard<std::mutex> g(ix->mu);
    BM25_TRY(rescore_index(ix, global_df, global_n_docs, global_n_tokens,
                           (cudaStream_t)cuda_stream));
    ix->doc_offset = doc_id_offset;
    return BM25_OK;
}

int bm25_index_shard_info(const bm25_index* ix, int64_t* doc_id_offset, int64_t* global_n_docs,
                          int64_t* global_n_tokens)
{
    clear_error();
    if (!ix)
        return set_error(BM25_E_INVALID, "index is NULL");
    if (doc_id_offset) *doc_id_offset = ix->doc_offset;
    if (global_n_docs) *global_n_docs = ix->stat_docs;
    if (global_n_tokens) *global_n_tokens = ix->stat_tokens;
    return BM25_OK;
}

int bm25_merge_topk(const int32_t* cand_ids, const float* cand_scores, int32_t n_shards,
                    int32_t n_queries, int32_t k, int32_t* out_ids, float* out_scores,
                    void* cuda_stream)
{
    clear_error();
    if (n_shards < 1 || n_queries < 0 || k < 1 || k > BM25_MAX_K ||
        (int64_t)n_shards * k > (int64_t)INT32_MAX)
        return set_error(BM25_E_INVALID, "need n_shards >= 1, n_queries >= 0, 1 <= k <= %d "
                         "(got %d, %d, %d)", BM25_MAX_K, n_shards, n_queries, k);
    if (n_queries > 0 && (!cand_ids || !cand_scores || !out_ids || !out_scores))
        return set_error(BM25_E_INVALID, "NULL argument");
    return merge_topk_device(cand_ids, cand_scores, n_shards, n_queries, k, out_ids, out_scores,
                             (cudaStream_t)cuda_stream);
}

int bm25_debug_set_handshake_polls(int32_t polls)
{
    clear_error();
    g_handshake_polls.store(polls < 0 ? kHandshakePolls : polls, std::memory_order_relaxed);
    return BM25_OK;
}

int bm25_debug_fail_allocs(int32_t n)
{
    clear_error();
    g_fail_allocs.store(n > 0 ? n : 0, std::memory_order_relaxed);
    return BM25_OK;
}

int bm25_index_set_plan(bm25_index* ix, const bm25_plan* plan)
{
    clear_error();
    if (!ix || !plan)
        return set_error(BM25_E_INVALID, "NULL argument");
    Plan p;
    BM25_TRY(merge_plan(plan, plan_of(ix), &p));
    std::lock_guard<std::mutex> g(ix->mu);
    ix->plan = p;
    return BM25_OK;
}

int bm25_index_get_plan(const bm25_index* ix, bm25_plan* plan)
{
    clear_error();
    if (!ix || !plan)
        return set_error(BM25_E_INVALID, "NULL argument");
    Plan p = plan_of(ix);
    plan->accumulator = p.accumulator;
    plan->tile_docs = p.tile_docs;
    plan->block_threads = p.threads;
    plan->dense_max_postings = p.dense_max;
    plan->stage_entries = p.stage_entries;
    plan->stages = p.stages;
    return BM25_OK;
}

}  // extern "C"
