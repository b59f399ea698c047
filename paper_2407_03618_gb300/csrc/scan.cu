// Device-wide exclusive prefix sum of uint32 (reduce-then-scan, three
// kernels, no inter-block waiting).  Used for the radix-sort digit offsets,
// the run (nnz) offsets of the CSC build and nothing else.
#include "device.cuh"
#include "internal.h"

namespace bm25 {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanIpt = 8;
constexpr int kScanTile = kScanThreads * kScanIpt;  // 2048 elements per block

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              int64_t n, uint32_t* block_sums)
{
    __shared__ uint32_t buf[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanIpt; i++) {
        int64_t p = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (p < n)
            s += in[p];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0)
        buf[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = (threadIdx.x < kScanThreads / 32) ? buf[threadIdx.x] : 0u;
        w = warp_sum(w);
        if (threadIdx.x == 0)
            block_sums[blockIdx.x] = w;
    }
}

// One block: exclusive scan of the block sums in place; total to *d_total.
__global__ void __launch_bounds__(1024) k_scan_spine(uint32_t* sums, int64_t n, uint32_t* d_total)
{
    __shared__ uint32_t buf[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t p = base + threadIdx.x;
        uint32_t v = (p < n) ? sums[p] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_sum(v, buf, &tot);
        if (p < n)
            sums[p] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0)
        *d_total = carry;
}

// Each block scans its 2048 elements (blocked: thread t owns 8 consecutive)
// and adds the block's offset.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* in, uint32_t* out,
                                                             int64_t n,
                                                             const uint32_t* __restrict__ offs)
{
    __shared__ uint32_t tile[kScanTile];
    __shared__ uint32_t buf[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanIpt; i++) {
        int64_t p = base + (int64_t)i * kScanThreads + threadIdx.x;
        tile[i * kScanThreads + threadIdx.x] = (p < n) ? in[p] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanIpt];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanIpt; i++) {
        v[i] = tile[threadIdx.x * kScanIpt + i];
        s += v[i];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_sum(s, buf, &tot) + offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanIpt; i++) {
        tile[threadIdx.x * kScanIpt + i] = run;
        run += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanIpt; i++) {
        int64_t p = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (p < n)
            out[p] = tile[i * kScanThreads + threadIdx.x];
    }
}

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                       uint32_t* tmp, cudaStream_t stream)
{
    if (n <= 0) {
        BM25_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), stream));
        return BM25_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    {
        ProfileScope ps_("k_scan_reduce", stream);
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, tmp);
    }
    {
        ProfileScope ps_("k_scan_spine", stream);
        k_scan_spine<<<1, 1024, 0, stream>>>(tmp, nb, d_total);
    }
    {
        ProfileScope ps_("k_scan_apply", stream);
        k_scan_apply<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, out, n, tmp);
    }
    count_launch(3);
    BM25_LAUNCH_CHECK();
    return BM25_OK;
}

}  // namespace bm25
