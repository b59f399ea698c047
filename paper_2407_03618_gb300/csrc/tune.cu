// Plan autotuner: times retrieval of a sample batch under candidate plans and
// keeps the fastest as the index's plan.  A plan changes speed only, never
// results.  The paper has no counterpart (its retrieval is one SciPy slice and
// sum per query batch); the choices tuned are the ones this library adds:
//   - the doc-tile width W of the shared-memory path (smaller tiles: more
//     CTAs per SM but more (tile, query) items per query);
//   - the consumer warps per CTA of that path (fewer: less per-item work
//     spread over fewer warps, more issue slots per warp);
//   - the accumulator per query-length bucket: queries whose columns hold at
//     most dense_max postings take the dense path, the rest the tiled path.
// The top-k radix width is fixed at 8-bit digits (one 256-bin histogram per
// pass, aggregated per warp) and is not tuned.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "internal.h"

using namespace bm25;

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer()
    {
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
    }
};

// Best of two timed calls after one untimed call (which also grows the
// workspace to the plan's needs).
int time_plan(const bm25_index* ix, bm25_workspace* ws, const int32_t* qt, int64_t n_tok,
              const int64_t* qo, int32_t nq, int32_t k, int32_t* ids, float* scores,
              const Plan& p, cudaStream_t s, Timer& t, double* ms)
{
    BM25_TRY(retrieve_device(ix, ws, qt, qo, nq, n_tok, nullptr, k, ids, scores, p, s));
    double best = DBL_MAX;
    for (int r = 0; r < 2; r++) {
        BM25_CUDA_TRY(cudaEventRecord(t.a, s));
        BM25_TRY(retrieve_device(ix, ws, qt, qo, nq, n_tok, nullptr, k, ids, scores, p, s));
        BM25_CUDA_TRY(cudaEventRecord(t.b, s));
        BM25_CUDA_TRY(cudaEventSynchronize(t.b));
        float e = 0.0f;
        BM25_CUDA_TRY(cudaEventElapsedTime(&e, t.a, t.b));
        best = std::min(best, (double)e);
    }
    *ms = best;
    return BM25_OK;
}

}  // namespace

extern "C" int bm25_autotune(bm25_index* ix, const int32_t* query_tokens, int64_t n_query_tokens,
                             const int64_t* query_offsets, int32_t n_queries, int32_t k,
                             void* cuda_stream, bm25_plan* best, double* best_ms,
                             bm25_plan* tried, double* tried_ms, int32_t tried_cap,
                             int32_t* n_tried)
{
    clear_error();
    if (!ix || !best)
        return set_error(BM25_E_INVALID, "NULL argument");
    if (n_queries < 1 || n_query_tokens < 0 || !query_offsets ||
        (n_query_tokens > 0 && !query_tokens))
        return set_error(BM25_E_INVALID, "autotuning needs a non-empty sample batch");
    if (k < 1 || (k < ix->n_docs ? k : ix->n_docs) > BM25_MAX_K)
        return set_error(BM25_E_INVALID, "k = %d outside [1, BM25_MAX_K]", k);
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ix->device)
        return set_error(BM25_E_INVALID, "current device is not the index's device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Plan base;
    {
        std::lock_guard<std::mutex> g(ix->mu);
        base = ix->plan;
    }
    DeviceInfo di;
    BM25_TRY(device_info(&di));

    Timer t;
    BM25_CUDA_TRY(cudaEventCreate(&t.a));
    BM25_CUDA_TRY(cudaEventCreate(&t.b));
    int32_t* ids = nullptr;
    float* scores = nullptr;
    const size_t n_out = (size_t)n_queries * (size_t)k;
    BM25_CUDA_TRY(cudaMalloc((void**)&ids, n_out * sizeof(int32_t)));
    if (cudaMalloc((void**)&scores, n_out * sizeof(float)) != cudaSuccess) {
        cudaFree(ids);
        return set_error(BM25_E_OOM, "output allocation failed");
    }
    bm25_workspace ws;
    ws.device = dev;

    std::vector<std::pair<Plan, double>> log;
    Plan cur = base;
    double cur_ms = DBL_MAX;
    constexpr double kMinGain = 0.01;
    int rc = BM25_OK;
    auto trial = [&](const Plan& p) {
        if (rc != BM25_OK)
            return;
        double ms = 0.0;
        int r = time_plan(ix, &ws, query_tokens, n_query_tokens, query_offsets, n_queries, k, ids,
                          scores, p, s, t, &ms);
        if (r == BM25_E_INVALID) {  // the plan does not fit this corpus / device: skip it
            clear_error();
            return;
        }
        if (r != BM25_OK) {
            rc = r;
            return;
        }
        log.emplace_back(p, ms);
        // a later candidate must be faster by more than kMinGain: timing
        // noise then leaves the plan where it is (each step tries the
        // library's default first)
        if (ms < cur_ms * (1.0 - kMinGain)) {
            cur_ms = ms;
            cur = p;
        }
    };
    const Plan def;  // the library's defaults
    auto default_first = [](std::vector<int32_t> v, int32_t d) {
        std::stable_partition(v.begin(), v.end(), [d](int32_t x) { return x == d; });
        return v;
    };
    // 1. the tile width, every query on the tiled path
    for (int32_t W : default_first({6144, 7168, 8192, 10240, 12288}, def.tile_docs)) {
        Plan p = base;
        p.accumulator = BM25_ACC_SMEM_TILED;
        p.tile_docs = W;
        p.threads = def.threads;
        p.stage_entries = def.stage_entries;
        p.stages = def.stages;
        trial(p);
    }
    // 1b. the consumer threads per CTA at that width
    const Plan width = cur;
    for (int32_t th : {128, 192, 256, 512}) {
        if (th == def.threads)
            continue;  // tried in step 1
        Plan p = width;
        p.threads = th;
        trial(p);
    }
    // 1c. the staging ring (buffer size x count) with those
    const Plan threads = cur;
    for (auto ring : {std::make_pair(512, 2), std::make_pair(1024, 2), std::make_pair(1024, 3),
                      std::make_pair(1536, 2), std::make_pair(2048, 2)}) {
        if (ring.first == threads.stage_entries && ring.second == threads.stages)
            continue;  // the ring the earlier steps ran with
        Plan p = threads;
        p.stage_entries = ring.first;
        p.stages = ring.second;
        trial(p);
    }
    // 2. the dense-path bound with that tile width
    const Plan tiled = cur;
    for (int32_t dmax : default_first({2048, 4096, 8192, 16384, 32768}, def.dense_max)) {
        Plan p = tiled;
        p.accumulator = BM25_ACC_AUTO;
        p.dense_max = dmax;
        trial(p);
    }
    workspace_release(&ws);
    cudaFree(ids);
    cudaFree(scores);
    if (rc != BM25_OK)
        return rc;
    if (log.empty())
        return set_error(BM25_E_INVALID, "no candidate plan fits this index on this device");
    {
        std::lock_guard<std::mutex> g(ix->mu);
        ix->plan = cur;
    }
    auto to_c = [](const Plan& p, bm25_plan* o) {
        o->accumulator = p.accumulator;
        o->tile_docs = p.tile_docs;
        o->block_threads = p.threads;
        o->dense_max_postings = p.dense_max;
        o->stage_entries = p.stage_entries;
        o->stages = p.stages;
    };
    to_c(cur, best);
    if (best_ms)
        *best_ms = cur_ms;
    if (n_tried)
        *n_tried = (int32_t)log.size();
    for (int32_t i = 0; tried && tried_ms && i < tried_cap && i < (int32_t)log.size(); i++) {
        to_c(log[i].first, &tried[i]);
        tried_ms[i] = log[i].second;
    }
    return BM25_OK;
}
