// Retrieval for callers that cannot allocate device memory.
//
// bm25_retrieve keeps its scratch in a workspace that grows with cudaMalloc
// on demand.  Some callers cannot allow that: a real-time serving loop with a
// fixed memory budget (cudaMalloc may synchronise the device and stall every
// stream), a process whose device memory is owned by another allocator that
// has taken all of it, or one that must not grow its footprint after start.
// bm25_retrieve_noalloc runs the same kernels with their scratch carved from
// one file-scope device array of kScratchBytes, so a call allocates nothing.
// Every GPU that loads this library holds that array for the life of the
// process.  It still calls the CUDA runtime (launches, a memset), so it must
// not be called from inside a CUDA host function or stream callback, where
// CUDA calls are not allowed.
//
// The array's device address is looked up once per device and kept; after a
// cudaDeviceReset the module is loaded again and the kept address is stale,
// so the library must not be used across a device reset.
//
// The array is shared by every call: calls that overlap on the GPU (on
// different streams, or from different threads) race on it and must be
// serialised by the caller.  The kernels write every scratch word they read
// within a call (the per-query threshold is reset by the first kernel), so
// the previous call's contents never leak into a result.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace bm25 {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kAlign = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_dev_ptr[64] = {};  // the array's device address, per device

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of the array on the current device.  cudaGetSymbolAddress
// returns it once the module is loaded on that device; the host-side symbol
// itself is not a device address and must never reach a kernel.
int scratch_ptr(int dev, void** out)
{
    if (dev < 0 || dev >= 64)
        return set_error(BM25_E_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(BM25_E_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                             cudaGetErrorString(e));
        g_dev_ptr[dev] = p;
    }
    *out = g_dev_ptr[dev];
    return BM25_OK;
}

}  // namespace
}  // namespace bm25

using namespace bm25;

extern "C" int bm25_retrieve_noalloc(const bm25_index* ix, const int32_t* query_tokens,
                                     int64_t n_query_tokens, const int64_t* query_offsets,
                                     int32_t n_queries, int32_t k, int32_t* out_ids,
                                     float* out_scores, void* cuda_stream)
{
    clear_error();
    BM25_TRY(check_retrieve_args(ix, n_query_tokens, n_queries, k));
    const int64_t N = ix->n_docs;
    const int64_t kp = k < N ? k : N;
    int dev = ix->device;
    if (n_queries == 0)
        return BM25_OK;

    Plan plan;
    {
        std::lock_guard<std::mutex> g(const_cast<bm25_index*>(ix)->mu);
        plan = ix->plan;
    }
    plan.accumulator = BM25_ACC_SMEM_TILED;  // the dense path needs vectors of N accumulators
    // the doc-tile geometry retrieve_device derives from the plan
    const int64_t W = tile_width(plan, N);
    const int64_t n_tiles = (N + W - 1) / W;

    const size_t b_q = align_up(query_arrays_bytes(n_queries));
    const size_t b_seg = align_up(sizeof(int32_t) * (size_t)n_query_tokens * (size_t)(n_tiles + 1));
    const size_t b_tcount = align_up(sizeof(uint32_t) * (size_t)n_queries * (size_t)n_tiles);
    const size_t b_cand =
        align_up(sizeof(unsigned long long) * (size_t)n_queries * (size_t)n_tiles * (size_t)kp);
    const size_t need = b_q + b_seg + b_tcount + b_cand;
    if (need > kScratchBytes)
        return set_error(BM25_E_INVALID,
                         "this batch needs %zu bytes of scratch; bm25_retrieve_noalloc holds %zu "
                         "(use fewer queries, tokens or a smaller k per call, or bm25_retrieve)",
                         need, kScratchBytes);

    void* base = nullptr;
    BM25_TRY(scratch_ptr(dev, &base));
    unsigned char* p = static_cast<unsigned char*>(base);
    // A workspace whose buffers are slices of the array and whose capacities
    // match this call exactly, so retrieve_device finds nothing to grow.
    bm25_workspace ws;
    ws.device = dev;
    ws.fixed = true;
    carve_queries(&ws, p, n_queries);
    p += b_q;
    ws.seg = reinterpret_cast<int32_t*>(p);
    ws.seg_cap = (size_t)n_query_tokens * (size_t)(n_tiles + 1);
    ws.tcount = reinterpret_cast<uint32_t*>(p + b_seg);
    ws.tcount_cap = (size_t)n_queries * (size_t)n_tiles;
    ws.cand = reinterpret_cast<unsigned long long*>(p + b_seg + b_tcount);
    ws.cand_cap = (size_t)n_queries * (size_t)n_tiles * (size_t)kp;
    ws.owns_staging = false;
    int rc = retrieve_device(ix, &ws, query_tokens, query_offsets, n_queries, n_query_tokens,
                             nullptr, k, out_ids, out_scores, plan, (cudaStream_t)cuda_stream);
    // the slices belong to the array: nothing is released
    return rc;
}
